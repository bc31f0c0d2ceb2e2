"""Failure paths exercised without a GPU fault: an HBM budget that refuses a
scratch allocation, a bounded device wait that runs out (a barrier nothing
completes), a full serving queue and a serving group larger than the
serving budget.  Each returns an error status and leaves
the context usable."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    import paper_2410_01231_gb300 as pg
    return pg


def _points(n):
    D, _, _ = synthetic.workload(1, n=n, nq=1)
    return D


def test_budget_refuses_scratch_and_context_stays_usable(pg):
    D = _points(3000)
    Dd = torch.from_numpy(D).cuda()
    small = pg.Context(hbm_budget_bytes=4096)
    with pytest.raises(pg.PGError) as e:
        pg.build_knn(small, Dd, 16)
    assert e.value.status == 6  # PG_ERR_BUDGET
    with pytest.raises(pg.PGError) as e:
        pg.Index.build_rng(small, Dd, K=16, L=32, R=16, iters=1)
    assert e.value.status == 6
    roomy = pg.Context(hbm_budget_bytes=1 << 30)
    ids, _ = pg.build_knn(roomy, Dd, 16)
    oi, _ = oracle.knn(D, 16)
    assert (ids.cpu().numpy() == oi).all()


def test_bounded_wait_expires_with_a_status(pg):
    ctx = pg.Context()
    with pytest.raises(pg.PGError) as e:
        ctx.selftest_wait_timeout(0.2)
    assert e.value.status == 4  # PG_ERR_TIMEOUT
    # the error word was consumed and the context still runs kernels
    D = _points(2000)
    ids, _ = pg.build_knn(ctx, torch.from_numpy(D).cuda(), 8, precision="bf16")
    oi, _ = oracle.knn(D, 8)
    assert (ids.cpu().numpy() == oi).all()
    ctx.sync()


def test_full_serving_queue_refuses_admission(pg):
    ctx = pg.Context()
    D = _points(3000)
    X = synthetic.inserts(1, 12000)
    idx = pg.Index.build_nswg(ctx, torch.from_numpy(D).cuda(), metric="l2", K=24, L=48, R=32,
                              M=16, alpha_deg=70.0, iters=1, seed=5)
    idx.reserve(3000 + 12000)
    srv = pg.Server(idx)
    srv.set_queue_limit(1)
    t = srv.submit_insert(X, 32)  # pending until the worker finishes it
    with pytest.raises(pg.PGError) as e:
        srv.submit_query(D[:4], 5, 16)
    assert e.value.status == 5  # PG_ERR_CAPACITY: admission refused
    assert srv.wait(t, 120.0)
    srv.set_queue_limit(0)
    t2, ids, _ = srv.submit_query(D[:4], 5, 16)
    assert srv.wait(t2, 60.0)
    srv.stop()
    assert ids.shape == (4, 5) and (ids[:, 0] >= 0).all()


def test_serving_budget_refuses_a_group_that_never_fits(pg):
    ctx = pg.Context()
    D = _points(2000)
    idx = pg.Index.build_nswg(ctx, torch.from_numpy(D).cuda(), metric="l2", K=16, L=32, R=16,
                              M=16, alpha_deg=70.0, iters=1, seed=4)
    srv = pg.Server(idx, max_batch=65536, slots=2)
    # a query row costs 4 d + 8 k + 12 bytes (604 for d = 128, k = 10):
    # 4,000 rows need 2,416,000 bytes, more than 1 MiB; 64 rows need 38,656
    srv.set_budget(1 << 20)
    big = np.ascontiguousarray(np.resize(D, (4000, D.shape[1])))
    t1, _, _ = srv.submit_query(big, 10, 32, 1)
    t2, ids, _ = srv.submit_query(D[:64], 10, 16, 1)
    with pytest.raises(pg.PGError) as e:
        srv.wait(t1, 60.0)
    assert e.value.status == 6  # PG_ERR_BUDGET
    assert srv.wait(t2, 60.0) and (ids[:, 0] >= 0).all()
    srv.set_budget(0)
    t3, ids3, _ = srv.submit_query(big, 10, 32, 1)
    assert srv.wait(t3, 120.0) and (ids3[:, 0] >= 0).all()
    srv.stop()

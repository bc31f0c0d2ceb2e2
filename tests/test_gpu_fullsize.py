"""Parity at the benchmark's full size (1M x 128 byte-valued mixture, K=64,
L=200, R=32), in the configuration bench.py times, on sampled outputs the
oracle computes one by one; and the spatially ordered tensor-core kNN on a
mid-size case."""
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


@pytest.fixture(scope="module")
def ctx(pg):
    return pg.Context()


def test_knn_bf16_spatial_order_matches_oracle_rows(ctx, pg):
    D, _ = synthetic.mixture_int(40000, 128, 40, 77)
    gi, gd = pg.build_knn(ctx, torch.from_numpy(D).cuda(), 64, precision="bf16")
    fi, fd = pg.build_knn(ctx, torch.from_numpy(D).cuda(), 64, precision="fp32")
    assert torch.equal(gi, fi) and torch.equal(gd, fd)
    rows = np.random.default_rng(3).choice(40000, 200, replace=False)
    oi, od = oracle.knn(D, 64, rows=rows)
    assert (gi.cpu().numpy()[rows] == oi).all()
    assert (gd.cpu().numpy()[rows] == od.astype(np.float32)).all()


@pytest.fixture(scope="module")
def full():
    D, Q, w = synthetic.workload(2)
    return D, Q, w


def test_full_size_steps_match_oracle_on_sampled_rows(ctx, pg, full):
    D, Q, w = full
    n, K, L, R = w["n"], w["K"], w["L"], w["R"]
    Dd = torch.from_numpy(D).cuda()
    rows = np.random.default_rng(11).choice(n, 48, replace=False)
    # a1: exact kNN graph (tensor-core form, as the bench runs it)
    gi, _ = pg.build_knn(ctx, Dd, K, precision="bf16")
    oi, _ = oracle.knn(D, K, rows=rows)
    gih = gi.cpu().numpy()
    assert (gih[rows] == oi).all()
    # a3: alpha-pruning of those rows given the same candidate lists
    off = torch.arange(n + 1, dtype=torch.int64, device="cuda") * K
    n1, d1 = pg.prune(ctx, Dd, off, gi.reshape(-1), R, 66.0)
    sub_off = np.zeros(n + 1, np.int64)
    cnts = np.zeros(n, np.int64)
    cnts[rows] = K
    sub_off[1:] = np.cumsum(cnts)
    sub_cand = np.concatenate([gih[u] for u in sorted(rows)]).astype(np.int32)
    on, od = oracle.prune(D, sub_off, sub_cand, R, 66.0)
    n1h, d1h = n1.cpu().numpy(), d1.cpu().numpy()
    assert (d1h[rows] == od[rows]).all() and (n1h[rows] == on[rows]).all()
    # a4: reverse union of the whole pass-1 graph, re-pruned rows
    uo, ui = pg.reverse_union(ctx, n1, d1)
    n2, d2 = pg.prune(ctx, Dd, uo, ui, R, 66.0)
    uoh, uih = uo.cpu().numpy(), ui.cpu().numpy()
    src = np.repeat(np.arange(n), d1h)
    dst = n1h[n1h >= 0]
    for u in rows[:8]:
        want = sorted(n1h[u, : d1h[u]].tolist() + src[dst == u].tolist())
        assert sorted(uih[uoh[u]: uoh[u + 1]].tolist()) == want
    urows = [uih[uoh[u]: uoh[u + 1]] for u in sorted(rows)]
    cnts = np.zeros(n, np.int64)
    cnts[np.sort(rows)] = [len(x) for x in urows]
    uoff = np.zeros(n + 1, np.int64)
    uoff[1:] = np.cumsum(cnts)
    on2, od2 = oracle.prune(D, uoff, np.concatenate(urows).astype(np.int32), R, 66.0)
    n2h, d2h = n2.cpu().numpy(), d2.cpu().numpy()
    assert (d2h[rows] == od2[rows]).all() and (n2h[rows] == on2[rows]).all()
    # a5: connectivity makes every node reachable (exactness is tested at 10k)
    ep = pg.medoid(ctx, Dd)
    pg.connect(ctx, Dd, n2, d2, ep)
    assert int(d2.max()) <= R
    # a6: self-search candidates of sampled rows equal the oracle's searches
    cand = pg.acquire_candidates(ctx, Dd, n2, d2, L).cpu().numpy()
    n2h, d2h = n2.cpu().numpy(), d2.cpu().numpy()
    ids, _ = oracle.search(D, n2h, d2h, D[rows[:16]], rows[:16], L, L)
    for i, u in enumerate(rows[:16]):
        want = [v for v in ids[i] if v != u and v >= 0]
        got = [v for v in cand[u] if v >= 0]
        assert got == want


def test_full_size_build_recall(ctx, pg, full):
    D, Q, w = full
    Dd = torch.from_numpy(D).cuda()
    idx = pg.Index.build_rng(ctx, Dd, K=w["K"], L=w["L"], R=w["R"], M=16, precision="bf16")
    qs = slice(0, 300)
    ids, dist = idx.search(torch.from_numpy(Q[qs]).cuda(), 10, 64)
    gt = oracle.knn(D, 10, Q=Q[qs])
    assert oracle.recall_at_k(ids.cpu().numpy(), Q[qs], D, 10, gt=gt) >= 0.95
    # returned distances are the exact squared distances
    got = dist.cpu().numpy()[:20, :3]
    for i in range(20):
        for j in range(3):
            v = int(ids[i, j])
            assert got[i, j] == np.float32(oracle.dist(Q[i], D[v]))

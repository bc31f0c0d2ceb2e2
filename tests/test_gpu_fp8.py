"""FP8-screened queries on the device path.

The FP8 rows (pg_encode_fp8) equal the oracle's E4M3 encoding bit for bit
(codes and scales).  Screened searches
return, for each query, ids sorted by (s, id) whose distances are the FP32
distances of those ids (within 1e-5 of the oracle's FP64 values, relative
to the scale of the data), with recall close to the FP32 search's; the
serving loop gives the same results as direct screened searches, and points
inserted into the index are found by screened searches.
"""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


@pytest.mark.parametrize("n,d", [(300, 128), (257, 96), (64, 20)])
def test_fp8_rows_equal_the_oracle_encoding(ctx, pg, n, d):
    rs = np.random.default_rng(n + d)
    D = rs.normal(0, 1, (n, d)).astype(np.float32)
    D[5] = 0.0                                   # zero row: scale 1, all codes 0
    D[6] = rs.integers(-3, 4, d).astype(np.float32) * 2.0 ** -12  # tiny values
    D[7, :] = 1.0
    D[7, 0] = -448.0 * 3                         # saturating magnitude
    codes, scale = pg.encode_fp8(ctx, dev(D))
    oc, osc = oracle.fp8_rows(D)
    assert (host(scale) == osc).all()
    assert (host(codes) == oc).all()


def _exact_s(D, Q, ids, metric):
    x = D[np.maximum(ids, 0)].astype(np.float64)
    q = Q.astype(np.float64)[:, None, :]
    if metric == "l2":
        return ((x - q) ** 2).sum(-1)
    return np.maximum(2.0 - 2.0 * (x * q).sum(-1), 0.0)


def _check_rows(ids, s, D, Q, metric, scale):
    assert (ids >= 0).all()
    # sorted by (s, id)
    for a, b in zip(range(ids.shape[1] - 1), range(1, ids.shape[1])):
        ok = (s[:, a] < s[:, b]) | ((s[:, a] == s[:, b]) & (ids[:, a] < ids[:, b]))
        assert ok.all()
    # distances are the FP32 distances of the returned ids
    ex = _exact_s(D, Q, ids, metric)
    assert (np.abs(s - ex) <= 1e-5 * scale).all()


def test_fp8_screened_queries_on_the_sphere(ctx, pg):
    """Unit rows of a 384-d sphere mixture, inner product (the serving recipe)."""
    D, Q, w = synthetic.workload(5, n=12000, nq=150)
    idx = pg.Index.build_nswg(ctx, dev(D), metric="ip", K=32, L=64, R=32, M=16, iters=1,
                              precision="bf16")
    gt = oracle.knn(D, 10, "ip", Q=Q)
    res = {}
    for prec in ("fp32", "fp8"):
        ids, s = idx.search(dev(Q), 10, 64, precision=prec)
        ids, s = host(ids), host(s)
        _check_rows(ids, s, D, Q, "ip", 4.0)
        res[prec] = oracle.recall_at_k(ids, Q, D, 10, "ip", gt=gt)
    assert res["fp8"] >= 0.85 and res["fp8"] >= res["fp32"] - 0.03, res


def test_fp8_screened_queries_narrow_rows(ctx, pg):
    """Rows of 36 elements (not a multiple of 16: four codes per load)."""
    D = synthetic.unit_gaussian(3000, 36, 21)
    Q = synthetic.unit_gaussian(100, 36, 22)
    idx = pg.Index.build_nswg(ctx, dev(D), metric="cosine", K=24, L=48, R=24, M=16, iters=1)
    gt = oracle.knn(D, 10, "cosine", Q=Q)
    res = {}
    for prec in ("fp32", "fp8"):
        ids, s = idx.search(dev(Q), 10, 64, precision=prec)
        ids, s = host(ids), host(s)
        _check_rows(ids, s, D, Q, "cosine", 4.0)
        res[prec] = oracle.recall_at_k(ids, Q, D, 10, "cosine", gt=gt)
    assert res["fp8"] >= 0.8 and res["fp8"] >= res["fp32"] - 0.05, res


def test_fp8_screened_queries_on_integer_rows(ctx, pg):
    """Byte-valued rows, squared L2: FP32 distances of the returned ids are
    exact integers, so they must equal the oracle's exactly."""
    D, Q, w = synthetic.workload(1, n=6000, nq=120)
    idx = pg.Index.build_rng(ctx, dev(D), K=20, L=64, R=24, iters=1, precision="bf16")
    gt = oracle.knn(D, 10, "l2", Q=Q)
    res = {}
    for prec in ("fp32", "fp8"):
        ids, s = idx.search(dev(Q), 10, 48, precision=prec)
        ids, s = host(ids), host(s)
        assert (s == _exact_s(D, Q, ids, "l2")).all()
        res[prec] = oracle.recall_at_k(ids, Q, D, 10, "l2", gt=gt)
    assert res["fp8"] >= 0.85 and res["fp8"] >= res["fp32"] - 0.03, res
    # host buffers give the same rows
    hi, hs = idx.search_host(Q, 10, 48, precision="fp8")
    di, ds = idx.search(dev(Q), 10, 48, precision="fp8")
    assert (hi == host(di)).all() and (hs == host(ds)).all()


def test_fp8_serving_and_insertion(ctx, pg):
    D, Q, _ = synthetic.workload(1, n=3600, nq=80)
    n0 = 3000
    ctx2 = pg.Context()
    idx = pg.Index.build_nswg(ctx2, dev(D[:n0]), metric="l2", K=24, L=48, R=32, M=16,
                              alpha_deg=70.0, iters=1, seed=6)
    idx.reserve(3600)
    # screened searches before the insertion make the FP8 rows of n0 points
    bi, bd = idx.search(dev(Q), 10, 48, upper_beam=4, precision="fp8")
    bi, bd = host(bi), host(bd)
    srv = pg.Server(idx, max_batch=64, slots=3)
    srv.set_precision("fp8")
    tq = [srv.submit_query(Q[i:i + 16], 10, 48, 4) for i in range(0, 80, 16)]
    ti = srv.submit_insert(D[n0:], 40, 4)
    # queries after the insertion: its points themselves, screened
    ta, ids_a, dist_a = srv.submit_query(D[n0:n0 + 40], 5, 48, 4)
    assert srv.wait_all([t for t, _, _ in tq] + [ti, ta], 120.0)
    srv.stop()
    # requests submitted before the insertion equal the searches made alone
    # on the index as it was then
    for i, (t, ids, dist) in zip(range(0, 80, 16), tq):
        assert (ids == bi[i:i + 16]).all() and (dist == bd[i:i + 16]).all()
    # inserted points are found: nearly every one returns itself first
    assert (dist_a[:, 0] == 0.0).mean() >= 0.95
    gi, gd = idx.search(dev(D[n0:n0 + 40]), 5, 48, upper_beam=4, precision="fp8")
    assert (host(gi) == ids_a).all() and (host(gd) == dist_a).all()

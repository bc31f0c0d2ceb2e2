"""kNN-graph refinement by 2-hop neighbours on the device (the KGraph /
NN-descent iteration of Section 3.1 as Exp. 12 describes it): equal to the
FP64 oracle's lists, which compare every 2-hop pair, on exact rows (so the
device's skipping of already-compared pairs changes nothing), for given and
drawn initial graphs; close to it on real rows; and a build that starts from
it keeps the framework's search quality (Exp. 12's observation)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu

M64 = (1 << 64) - 1


@pytest.fixture(scope="module")
def pg():
    import paper_2410_01231_gb300 as pg
    return pg


@pytest.fixture(scope="module")
def ctx(pg):
    return pg.Context()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _splitmix64(x):
    z = (x + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def _drawn(n, K, seed):
    """The library's initial draw written out (published SplitMix64)."""
    out = np.empty(n * K, np.int64)
    for t in range(n * K):
        out[t] = (_splitmix64(t ^ seed) * n) >> 64
    return out.reshape(n, K).astype(np.int32)


@pytest.mark.parametrize("K,iters", [(8, 0), (8, 3), (32, 2), (64, 4)])
def test_descent_equals_the_oracle_on_exact_rows(ctx, pg, K, iters):
    D, _, _ = synthetic.workload(1, n=2500, nq=1)
    init = np.random.default_rng(K + iters).integers(-1, 2500, size=(2500, K)).astype(np.int32)
    gi, gd, upd = pg.knn_descent(ctx, dev(D), K, iters, init=dev(init))
    oi, od = oracle.knn_descent(D, init, iters)
    assert (gi.cpu().numpy() == oi).all()
    m = oi >= 0
    assert (gd.cpu().numpy()[m] == od[m].astype(np.float32)).all()
    assert len(upd) == iters and all(u >= 0 for u in upd)


def test_descent_library_draw_equals_its_written_definition(ctx, pg):
    D, _, _ = synthetic.workload(1, n=700, nq=1)
    gi, _, upd = pg.knn_descent(ctx, dev(D), 16, 3, seed=12345)
    oi, _ = oracle.knn_descent(D, _drawn(700, 16, 12345), 3)
    assert (gi.cpu().numpy() == oi).all()
    assert upd[0] > upd[-1]


def test_descent_on_real_rows_follows_the_oracle(ctx, pg):
    D, _ = synthetic.mixture_float(2000, 48, 10, 61)
    init = np.random.default_rng(4).integers(0, 2000, size=(2000, 16)).astype(np.int32)
    gi, _, _ = pg.knn_descent(ctx, dev(D), 16, 4, init=dev(init))
    oi, _ = oracle.knn_descent(D, init, 4)
    same = (gi.cpu().numpy() == oi).all(1).mean()
    assert same >= 0.99, same
    gt, _ = oracle.knn(D, 16)
    rg = np.mean([len(set(gi.cpu().numpy()[u]) & set(gt[u])) for u in range(2000)]) / 16
    ro = np.mean([len(set(oi[u]) & set(gt[u])) for u in range(2000)]) / 16
    assert abs(rg - ro) <= 0.002


def test_build_from_the_descent_graph_keeps_search_quality(ctx, pg):
    """Exp. 12: the framework's iterations make up for an approximate initial
    KNNG; the build from a few 2-hop iterations reaches the search quality
    of the build from the exact kNN graph."""
    D, Q, w = synthetic.workload(1)
    Dd = dev(D)
    prm = dict(K=w["K"], L=w["L"], R=w["R"], M=16, iters=2)
    gt = oracle.knn(D, 10, Q=Q)
    rec = {}
    for it in (-1, 4):
        idx = pg.Index.build_rng(ctx, Dd, knn_descent_iters=it, **prm)
        ids, _ = idx.search(dev(Q), 10, 64)
        rec[it] = oracle.recall_at_k(ids.cpu().numpy(), Q, D, 10, gt=gt)
        _, nb, dg = idx.layer(0)
        assert (dg.cpu().numpy() <= w["R"]).all()
        idx.close()
    assert rec[4] >= rec[-1] - 0.02 and rec[-1] >= 0.95, rec
    with pytest.raises(pg.PGError):
        pg.Index.build_rng(ctx, Dd, knn_descent_iters=3, **dict(prm, K=80))

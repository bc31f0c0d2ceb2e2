"""Randomized parity of the CUDA path with the oracle on integer-valued rows
(where every distance is exact, so results must be identical): random sizes,
widths, K, pool widths and degree bounds."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle

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


def _rows(rng, n, d):
    hi = int(rng.choice([3, 16, 256]))
    return rng.integers(0, hi, size=(n, d)).astype(np.float32)


@pytest.mark.parametrize("seed", range(8))
def test_knn_random_shapes(ctx, pg, seed):
    rng = np.random.default_rng(2000 + seed)
    n = int(rng.integers(2, 3000))
    d = int(rng.choice([4, 16, 64, 128, 192]))
    K = int(rng.integers(1, 65))
    D = _rows(rng, n, d)
    oi, od = oracle.knn(D, K)
    for precision in ("fp32", "bf16"):
        gi, gd = pg.build_knn(ctx, dev(D), K, precision=precision)
        assert (host(gi) == oi).all(), precision
        m = oi >= 0
        assert (host(gd)[m] == od[m].astype(np.float32)).all(), precision


@pytest.mark.parametrize("seed", range(6))
def test_acquire_random_graphs(ctx, pg, seed):
    rng = np.random.default_rng(3000 + seed)
    n = int(rng.integers(20, 2500))
    d = int(rng.choice([16, 32, 128]))
    R = int(rng.integers(2, 33))
    L = int(rng.integers(1, 129))
    D = _rows(rng, n, d)
    K = min(n - 1, 24)
    ids, _ = oracle.knn(D, K)
    nbr, deg = oracle.prune(D, np.arange(n + 1, dtype=np.int64) * K, ids.ravel(), R, 66.0)
    ocand = oracle.acquire(D, nbr, deg, L)
    for precision in ("fp32", "bf16"):
        cand = pg.acquire_candidates(ctx, dev(D), dev(nbr), dev(deg), L, precision=precision)
        assert (host(cand) == ocand).all(), precision


@pytest.mark.parametrize("seed", range(6))
def test_connect_random_graphs(ctx, pg, seed):
    rng = np.random.default_rng(4000 + seed)
    n = int(rng.integers(10, 3000))
    d = int(rng.choice([16, 128]))
    R = int(rng.integers(4, 33))
    D = _rows(rng, n, d)
    K = min(n - 1, 8)
    ids, _ = oracle.knn(D, K)
    nbr, deg = oracle.prune(D, np.arange(n + 1, dtype=np.int64) * K, ids.ravel(), R, 60.0)
    ep = int(rng.integers(0, n))
    on, od, oadded = oracle.connect(D, nbr, deg, ep)
    gn, gdg = dev(nbr), dev(deg)
    if oadded < 0:  # no reached node with a free slot: both sides refuse
        with pytest.raises(pg.PGError) as e:
            pg.connect(ctx, dev(D), gn, gdg, ep)
        assert e.value.status == 5
        return
    gadded = pg.connect(ctx, dev(D), gn, gdg, ep)
    assert gadded == oadded
    assert (host(gdg) == od).all() and (host(gn) == on).all()

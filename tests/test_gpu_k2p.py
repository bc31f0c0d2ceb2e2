"""K2P (Section 5.4) on the device: pruning the next iteration's k-CNA lists
with the previous iteration's kept lists reused gives the lists of plain
pruning (and of the FP64 oracle) with fewer occlusion tests, in every
kernel path (byte rows held in registers, byte rows, FP32 rows with FP64
rechecks, the chord of unit rows); builds with and without the reuse give
the same graph."""
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


def _iteration(D, metric, K, R, L, alpha):
    """C1 = exact kNN rows, N1 = their pruning (the previous pass), and the
    next iteration's C2 (acquisition on the refined, connected graph), all
    from the oracle."""
    n = D.shape[0]
    C1, _ = oracle.knn(D, K, metric)
    off1 = np.arange(n + 1, dtype=np.int64) * K
    N1, deg1 = oracle.prune(D, off1, C1.ravel(), R, alpha, metric)
    uoff, uids = oracle.reverse_union(N1, deg1)
    G, gdeg = oracle.prune(D, uoff, uids, R, alpha, metric)
    G, gdeg, _ = oracle.connect(D, G, gdeg, oracle.medoid(D, metric), metric)
    C2 = oracle.acquire(D, G, gdeg, L, metric)
    return N1, deg1, C2


CASES = {
    "bytes_reg": (lambda: synthetic.workload(1, n=1500, nq=1)[0], "l2", "bf16", 16),
    "bytes_wide_r": (lambda: synthetic.workload(1, n=1500, nq=1)[0], "l2", "bf16", 48),
    "bytes_fp32": (lambda: synthetic.workload(1, n=1500, nq=1)[0], "l2", "fp32", 16),
    "float": (lambda: synthetic.mixture_float(1500, 64, 12, 41)[0], "l2", "fp32", 16),
    "cosine": (lambda: synthetic.unit_gaussian(1500, 48, 42), "cosine", "fp32", 16),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("alpha", [60.0, 66.0])
def test_k2p_equals_plain_pruning_and_the_oracle(ctx, pg, case, alpha):
    make, metric, precision, R = CASES[case]
    D = make()
    n, K, L = D.shape[0], 24, 48
    N1, deg1, C2 = _iteration(D, metric, K, R, L, alpha)
    off = np.arange(n + 1, dtype=np.int64) * L
    Dd = dev(D)
    pn, pd, ps = pg.prune(ctx, Dd, dev(off), dev(C2.ravel()), R, alpha, metric, precision,
                          stats=True)
    kn, kd, ks = pg.prune_k2p(ctx, Dd, dev(off), dev(C2.ravel()), dev(N1), dev(deg1), R, alpha,
                              metric, precision, stats=True)
    assert torch.equal(kd, pd) and torch.equal(kn, pn)
    on, od = oracle.prune(D, off, C2.ravel(), R, alpha, metric)
    assert (kd.cpu().numpy() == od).all() and (kn.cpu().numpy() == on).all()
    assert ks["edges"] == ps["edges"]
    assert ks["occlusion_tests"] < ps["occlusion_tests"], (ks, ps)


def test_k2p_with_a_previous_pass_at_a_smaller_angle(ctx, pg):
    """Lists kept at 60 degrees are a valid premise for pruning at 66: a pair
    that does not occlude at 60 does not occlude at any larger angle."""
    D = synthetic.workload(1, n=1200, nq=1)[0]
    n, K, L, R = D.shape[0], 24, 48, 16
    N1, deg1, C2 = _iteration(D, "l2", K, R, L, 60.0)
    off = np.arange(n + 1, dtype=np.int64) * L
    kn, kd = pg.prune_k2p(ctx, dev(D), dev(off), dev(C2.ravel()), dev(N1), dev(deg1), R, 66.0)
    on, od = oracle.prune(D, off, C2.ravel(), R, 66.0)
    assert (kd.cpu().numpy() == od).all() and (kn.cpu().numpy() == on).all()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_builds_with_and_without_reuse_give_the_same_graph(ctx, pg, precision):
    D, _, _ = synthetic.workload(1, n=6000, nq=1)
    Dd = dev(D)
    prm = dict(K=20, L=64, R=24, M=16, iters=2, precision=precision, route_layers=0)
    graphs, tests = [], []
    for reuse in (0, 1):
        ctx.set_timing(True)  # resets the device counters
        idx = pg.Index.build_rng(ctx, Dd, reuse_pruning=reuse, **prm)
        tests.append(ctx.counter("prune_occlusion_tests"))
        ctx.set_timing(False)
        _, nb, dg = idx.layer(0)
        graphs.append((nb.clone(), dg.clone()))
        idx.close()
    assert torch.equal(graphs[0][0], graphs[1][0]) and torch.equal(graphs[0][1], graphs[1][1])
    assert tests[1] < tests[0], tests

"""Quality examination on the device (Section 5.2, Theorem 3, Algorithm 6's
termination): r(u) of the k-CNA lists equals the FP64 oracle's on the same
sample, element by element, and so does the sampled estimate; a build with
a quality target stops at the first iteration whose estimate meets it, and
its graph is the fixed-iteration build's with that many iterations."""
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


DATA = {
    "bytes": (lambda: synthetic.workload(1, n=3000, nq=1)[0], "l2"),
    "float": (lambda: synthetic.mixture_float(2500, 64, 10, 51)[0], "l2"),
    "cosine": (lambda: synthetic.unit_gaussian(2500, 32, 52), "cosine"),
}


@pytest.mark.parametrize("kind", sorted(DATA))
@pytest.mark.parametrize("k", [1, 10, 32])
def test_kcna_recall_equals_the_oracle(ctx, pg, kind, k):
    make, metric = DATA[kind]
    D = make()
    n, K, R, L = D.shape[0], 16, 16, 40
    ids, _ = oracle.knn(D, K, metric)
    nbr, deg = oracle.prune(D, np.arange(n + 1, dtype=np.int64) * K, ids.ravel(), R, 66.0, metric)
    cand = oracle.acquire(D, nbr, deg, L, metric)
    # damage some rows: repeated ids, the point itself, padding
    rng = np.random.default_rng(5)
    for u in rng.choice(n, 60, replace=False):
        cand[u, 1] = cand[u, 0]
        cand[u, 2] = u
        cand[u, 3:6] = -1
    ns = oracle.quality_sample_size(n, 0.6)
    seed = 17
    sample = np.sort(np.random.default_rng(seed).choice(n, size=min(ns, n), replace=False))
    rec, mean = pg.kcna_recall(ctx, dev(D), dev(cand), k, dev(sample.astype(np.int32)), metric)
    want = oracle.kcna_recall(D, cand, k, metric, rows=sample)
    assert (rec.cpu().numpy() == want).all()
    assert mean == pytest.approx(oracle.estimate_quality(D, cand, k, ns, seed, metric), abs=1e-12)


def test_kcna_recall_rejects_bad_sample_ids(ctx, pg):
    D = synthetic.workload(1, n=500, nq=1)[0]
    cand = np.full((500, 8), -1, np.int32)
    with pytest.raises(pg.PGError) as e:
        pg.kcna_recall(ctx, dev(D), dev(cand), 4, dev(np.array([3, 500], np.int32)))
    assert e.value.status == 8


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_build_stops_when_the_estimate_meets_the_target(ctx, pg, precision):
    D, _, _ = synthetic.workload(1, n=8000, nq=1)
    Dd = dev(D)
    base = dict(K=16, L=48, R=24, M=16, precision=precision, route_layers=0)
    # a target the first iteration meets: one iteration only
    idx = pg.Index.build_rng(ctx, Dd, iters=4, quality_target=0.05, **base)
    its, ns, est = idx.quality()
    assert its == 1 and len(est) == 1 and est[0] >= 0.05
    assert ns == pg.quality_sample_size(8000, 0.6)
    _, nq1, dq1 = idx.layer(0)
    ref = pg.Index.build_rng(ctx, Dd, iters=1, **base)
    _, nr, dr = ref.layer(0)
    assert torch.equal(nq1, nr) and torch.equal(dq1, dr)
    assert ref.quality()[:2] == (1, 0)
    # the highest target: iterations run until an estimate reaches it (or all
    # of them have run), each estimate recorded
    idx2 = pg.Index.build_rng(ctx, Dd, iters=3, quality_target=1.0, **base)
    its2, _, est2 = idx2.quality()
    assert len(est2) == its2 and 1 <= its2 <= 3
    assert all(e < 1.0 for e in est2[:-1]) and (its2 == 3 or est2[-1] >= 1.0)
    assert est2[0] == est[0]  # the same sample and lists after the first iteration
    for x in (idx, ref, idx2):
        x.close()

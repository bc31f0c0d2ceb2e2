"""Quality examination (Section 5.2, Theorem 3) in the oracle, on CPU: the
sample size against hand-computed values of the bound and its minimality,
the concentration it promises checked by simulation, and r(u) / the sampled
estimator on exact, damaged and tied candidate lists."""
import math

import numpy as np
import pytest

import oracle
import synthetic


def test_sample_size_hand_values():
    # (8 + 1.2) * 1 * ln(10^6) / 0.36 = 353.06...  ->  354   (eps = 0.6, Section 6)
    assert oracle.quality_sample_size(10**6, 0.6, 1) == 354
    # (8 + 0.2) * 2 * ln(1000) / 0.01 = 11328.8...  ->  11329
    assert oracle.quality_sample_size(1000, 0.1, 2) == 11329
    # (8 + 0.4) * 1 * ln(5000) / 0.04 = 1788.6...  ->  1789
    assert oracle.quality_sample_size(5000, 0.2, 1) == 1789
    with pytest.raises(ValueError):
        oracle.quality_sample_size(1, 0.5)


@pytest.mark.parametrize("n,eps,l", [(10**6, 0.6, 1), (5000, 0.2, 1), (1000, 0.1, 2)])
def test_sample_size_is_the_smallest_meeting_the_proof_bound(n, eps, l):
    ns = oracle.quality_sample_size(n, eps, l)
    # the proof's tail bound with mu <= 1: exp(-eps^2 n_s / (8 + 2 eps)) <= n^-l
    tail = lambda m: math.exp(-eps * eps * m / (8 + 2 * eps))
    assert tail(ns) <= n ** -l < tail(ns - 1)


def test_sampled_mean_concentrates_as_promised():
    rs = np.random.default_rng(11)
    n, eps, l = 5000, 0.2, 1
    r = np.where(rs.random(n) < 0.7, 1.0, rs.integers(0, 10, n) / 10.0)
    mu = r.mean()
    ns = oracle.quality_sample_size(n, eps, l)
    fails = 0
    for _ in range(2000):
        s = rs.choice(n, size=ns, replace=False)
        fails += abs(r[s].mean() - mu) >= eps / 2
    assert fails == 0  # the bound allows 2000 * n^-1 = 0.4 in expectation
    # far below the bound the guarantee is visibly lost
    few = sum(abs(r[rs.choice(n, size=3, replace=False)].mean() - mu) >= eps / 2
              for _ in range(2000))
    assert few > 200


def test_recall_of_exact_damaged_and_tied_lists():
    D, _, _ = synthetic.workload(1, n=600, nq=1)
    k = 10
    ids, ds = oracle.knn(D, k)
    assert (oracle.kcna_recall(D, ids, k) == 1.0).all()
    # replacing entries by points beyond the k-th distance costs 1/k each
    far = np.argsort(-((D - D[0]) ** 2).sum(1))[:3]
    bad = ids.copy()
    bad[0, [1, 4, 7]] = far
    r = oracle.kcna_recall(D, bad, k)
    assert r[0] == pytest.approx(0.7) and (r[1:] == 1.0).all()
    # repeated ids, self and -1 count never or once
    bad[1, :3] = [ids[1, 0], ids[1, 0], 1]
    bad[2, 5] = -1
    r = oracle.kcna_recall(D, bad, k)
    assert r[1] == pytest.approx(0.8) and r[2] == pytest.approx(0.9)
    # a point at the k-th distance that is not in the exact list still counts:
    # on an integer grid the centre has 4 neighbours at distance 1, 4 at 2, ...
    g = np.array([(x, y, 0, 0) for x in range(7) for y in range(7)], np.float32)
    gi, gd = oracle.knn(g, 6)
    u = 24  # the centre (3, 3): neighbours 1 (x4) then 2 (x4); the 6th is a tie
    s = ((g.astype(np.float64) - g[u]) ** 2).sum(1)
    alt = [v for v in np.nonzero(s == gd[u, 5])[0] if v not in gi[u] and v != u]
    assert gd[u, 5] == 2.0 and alt
    t = gi.copy()
    t[u, 5] = alt[0]
    assert oracle.kcna_recall(g, t, 6, rows=[u])[0] == 1.0
    t[u, 5] = int(np.argmax(s))  # a corner, beyond the 6th distance
    assert oracle.kcna_recall(g, t, 6, rows=[u])[0] == pytest.approx(5 / 6)


def test_estimator_on_acquisition_lists():
    D, _, _ = synthetic.workload(1, n=2000, nq=1)
    nbr, deg, _ = oracle.build_rng(D, 16, 48, 16, 66.0, 60.0, 1, "l2")
    cand = oracle.acquire(D, nbr, deg, 48)
    k = 10
    full = oracle.kcna_recall(D, cand, k).mean()
    assert oracle.estimate_quality(D, cand, k, 2000, seed=1) == pytest.approx(full)
    ns = oracle.quality_sample_size(2000, 0.3, 1)
    assert abs(oracle.estimate_quality(D, cand, k, ns, seed=2) - full) < 0.15
    assert 0.5 < full <= 1.0

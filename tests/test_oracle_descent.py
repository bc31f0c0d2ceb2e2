"""The oracle's kNN-graph refinement by 2-hop neighbours (the KGraph
iteration of the initialization phase as Exp. 12 describes it), pinned on
CPU: a literal restatement with Python sets and exact integer distances,
the exact kNN graph is a fixed point, iteration 0 is the sorted initial
draw, the K-th distance of every row never grows, and on clustered data
the lists approach the exact kNN."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synthetic


def exact_s(x, y):
    return int(sum((int(a) - int(b)) ** 2 for a, b in zip(x, y)))


def _literal(D, init, iters):
    n, K = init.shape
    cur = []
    for u in range(n):
        ids = {int(v) for v in init[u] if 0 <= v < n and v != u}
        cur.append(sorted((exact_s(D[u], D[v]), v) for v in ids)[:K])
    for _ in range(iters):
        nxt = []
        for u in range(n):
            cand = set()
            for _, v in cur[u]:
                cand.add(v)
                cand.update(w for _, w in cur[v])
            cand.discard(u)
            nxt.append(sorted((exact_s(D[u], D[w]), w) for w in cand)[:K])
        cur = nxt
    ids = np.full((n, K), -1, np.int32)
    for u in range(n):
        for j, (_, v) in enumerate(cur[u]):
            ids[u, j] = v
    return ids


def _init(n, K, seed):
    return np.random.default_rng(seed).integers(0, n, size=(n, K)).astype(np.int32)


@pytest.mark.parametrize("seed", range(5))
def test_descent_equals_its_literal_statement(seed):
    rs = np.random.default_rng(seed)
    n, K, d = int(rs.integers(5, 70)), int(rs.integers(1, 9)), int(rs.integers(1, 5))
    D = rs.integers(0, 5, size=(n, d)).astype(np.float32)  # many exact ties
    init = _init(n, K, 50 + seed)
    for iters in (0, 1, 3):
        ids, _ = oracle.knn_descent(D, init, iters)
        assert (ids == _literal(D, init, iters)).all(), (seed, iters)


def test_exact_knn_is_a_fixed_point():
    D, _, _ = synthetic.workload(1, n=600, nq=1)
    ids, dist = oracle.knn(D, 12)
    out, od = oracle.knn_descent(D, ids, 3)
    assert (out == ids).all() and np.allclose(od, dist)


def test_kth_distance_never_grows_and_lists_approach_exact():
    D, _ = synthetic.mixture_int(1500, 32, 12, 3)
    K = 10
    init = _init(1500, K, 7)
    gt, gd = oracle.knn(D, K)
    prev, rec = None, []
    for it in range(6):
        ids, dist = oracle.knn_descent(D, init, it)
        kth = dist[:, -1]
        if prev is not None:
            assert (kth <= prev).all()
        prev = kth
        rec.append(np.mean([len(set(ids[u]) & set(gt[u])) / K for u in range(1500)]))
    assert rec[0] < 0.05 and rec[-1] > 0.9 and all(b >= a for a, b in zip(rec, rec[1:]))

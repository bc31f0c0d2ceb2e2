"""Pins for the FP64 oracle: each test checks it against something other than
itself (exact integer arithmetic, an independent geometric computation, a
literal reading of a printed algorithm, published constants, closed forms).
CPU only."""
from __future__ import annotations

import math
import os
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def int_data(n, d, seed, hi=16):
    rng = np.random.default_rng(seed)
    return rng.integers(0, hi, size=(n, d)).astype(np.float32)


def exact_s(x, y):
    """Squared L2 in exact integer arithmetic (integer-valued rows)."""
    return sum((int(a) - int(b)) ** 2 for a, b in zip(x, y))


# --------------------------------------------------------------------------
# distances
# --------------------------------------------------------------------------
def test_dist_l2_exact_on_integers():
    D = int_data(20, 37, 1, hi=256)
    for i in range(0, 20, 3):
        for j in range(20):
            assert oracle.dist(D[i], D[j]) == exact_s(D[i], D[j])


def test_dist_cosine_is_squared_chord():
    rng = np.random.default_rng(2)
    X = rng.normal(size=(30, 24))
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    X = X.astype(np.float32)
    for i in range(10):
        for j in range(30):
            c = oracle.dist(X[i], X[j], "cosine")
            e = float(np.sum((X[i].astype(np.float64) - X[j].astype(np.float64)) ** 2))
            assert abs(c - e) < 1e-6
        # 2 - 2|x|^2: float32 rows are unit only to rounding
        assert 0.0 <= oracle.dist(X[i], X[i], "cosine") < 1e-6


# --------------------------------------------------------------------------
# exact kNN: brute force in exact integer arithmetic, ties by id
# --------------------------------------------------------------------------
def test_knn_matches_exact_integer_bruteforce():
    D = int_data(150, 9, 3, hi=6)  # small range: many exact ties
    K = 12
    ids, ds = oracle.knn(D, K)
    for u in range(D.shape[0]):
        pairs = sorted((exact_s(D[u], D[v]), v) for v in range(D.shape[0]) if v != u)[:K]
        assert [v for _, v in pairs] == ids[u].tolist()
        assert [float(s) for s, _ in pairs] == ds[u].tolist()


def test_knn_external_queries_and_padding():
    D = int_data(7, 4, 4)
    Q = int_data(3, 4, 5)
    ids, ds = oracle.knn(D, 10, Q=Q)
    assert (ids[:, 7:] == -1).all() and np.isinf(ds[:, 7:]).all()
    for q in range(3):
        pairs = sorted((exact_s(Q[q], D[v]), v) for v in range(7))
        assert [v for _, v in pairs] == ids[q, :7].tolist()


# --------------------------------------------------------------------------
# alpha-pruning
# --------------------------------------------------------------------------
def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_prune_hand_worked_triangle():
    D = np.array([[0.0, 0.0], [1.0, 0.0], [1.2, 1.0]], np.float32)
    off = np.array([0, 2, 2, 2], np.int64)
    cand = np.array([2, 1], np.int32)
    for alpha, kept in _read_golden("prune_triangle_2d.txt"):
        nbr, deg = oracle.prune(D, off, cand, 4, float(alpha))
        want = [int(x) for x in kept.split(",")]
        assert nbr[0, : deg[0]].tolist() == want, alpha


def _angle_deg(u, w, v):
    a = np.asarray(u, np.float64) - np.asarray(w, np.float64)
    b = np.asarray(v, np.float64) - np.asarray(w, np.float64)
    return math.degrees(abs(math.atan2(a[0] * b[1] - a[1] * b[0], a[0] * b[0] + a[1] * b[1])))


def test_prune_angle_clause_against_atan2_geometry():
    """For random planar triangles where both distance clauses hold, v is
    pruned exactly when the angle at w (measured with atan2) exceeds alpha."""
    rng = np.random.default_rng(6)
    checked = 0
    for _ in range(3000):
        P = rng.uniform(-10, 10, size=(3, 2)).astype(np.float32)
        u, w, v = P
        suw, suv, svw = (oracle.dist(u, w), oracle.dist(u, v), oracle.dist(v, w))
        if not (suw < suv and svw < suv):
            continue
        ang = _angle_deg(u, w, v)
        alpha = float(rng.uniform(55, 125))
        if abs(ang - alpha) < 1e-6:
            continue
        off = np.array([0, 2, 2, 2], np.int64)
        nbr, deg = oracle.prune(P, off, np.array([2, 1], np.int32), 4, alpha)
        assert nbr[0, : deg[0]].tolist() == ([1] if ang > alpha else [1, 2])
        checked += 1
    assert checked > 500


def _literal_alg3(D, u, cand, M):
    """Algorithm 3 as printed: ascending dist(u,v); v dominated iff some
    selected w has dist(v,w) < dist(u,v); stop at M selected."""
    xs = D.astype(np.float64)
    order = sorted(set(c for c in cand if c != u),
                   key=lambda v: (np.linalg.norm(xs[u] - xs[v]), v))
    kept = []
    for v in order:
        dom = any(np.linalg.norm(xs[v] - xs[w]) < np.linalg.norm(xs[u] - xs[v]) for w in kept)
        if not dom:
            kept.append(v)
        if len(kept) >= M:
            break
    return kept


def test_prune_alpha60_equals_rng_algorithm3():
    """alpha = 60 degrees is RNG pruning (Section 4.2) on tie-free data."""
    rng = np.random.default_rng(7)
    D = rng.normal(size=(120, 6)).astype(np.float32)
    ids, _ = oracle.knn(D, 40)
    off = np.arange(121, dtype=np.int64) * 40
    for M in (5, 12, 40):
        nbr, deg = oracle.prune(D, off, ids.ravel(), M, 60.0)
        for u in range(120):
            assert nbr[u, : deg[u]].tolist() == _literal_alg3(D, u, ids[u].tolist(), M)


def test_prune_alpha180_keeps_first_R():
    """No triangle has an angle above 180 degrees, so alpha = 180 prunes
    nothing: the first min(R, |C|) distinct candidates by (s, id) stay."""
    rng = np.random.default_rng(8)
    D = rng.normal(size=(80, 5)).astype(np.float32)
    cand = rng.integers(-1, 80, size=(80, 30)).astype(np.int32)
    off = np.arange(81, dtype=np.int64) * 30
    nbr, deg = oracle.prune(D, off, cand.ravel(), 10, 180.0)
    for u in range(80):
        ok = sorted({(oracle.dist(D[u], D[v]), v) for v in cand[u] if v >= 0 and v != u})
        assert nbr[u, : deg[u]].tolist() == [v for _, v in ok[:10]]


def _exact_occludes(D, u, w, v, cos_a):
    """Occlusion decided in exact/high-precision arithmetic (integer rows)."""
    suw, suv, svw = exact_s(D[u], D[w]), exact_s(D[u], D[v]), exact_s(D[v], D[w])
    if not (suw < suv and svw < suv):
        return False, 0
    getcontext().prec = 60
    lhs = Decimal(suw + svw - suv)
    rhs = 2 * Decimal(cos_a) * (Decimal(suw) * Decimal(svw)).sqrt()
    # lhs is an exact integer; when it is 0 only the sign of rhs decides,
    # which FP64 reproduces exactly, so such decisions are never tight
    margin = Decimal(1) if lhs == 0 else abs(lhs - rhs) / Decimal(suw + svw + suv)
    return lhs < rhs, margin


@pytest.mark.parametrize("alpha", [60.0, 66.0, 75.0, 90.0])
def test_prune_output_is_the_defined_set(alpha):
    """Independent check of the definition on integer data with many ties:
    kept rows follow (s, id) order; no kept v is occluded by an earlier kept
    w; every skipped candidate before the stop is occluded by a kept w."""
    D = int_data(200, 8, 9, hi=5)
    rng = np.random.default_rng(10)
    cand = rng.integers(0, 200, size=(200, 60)).astype(np.int32)
    off = np.arange(201, dtype=np.int64) * 60
    R = 9
    cos_a = oracle.cos_alpha(alpha)
    nbr, deg = oracle.prune(D, off, cand.ravel(), R, alpha)
    ambiguous = 0
    for u in range(200):
        order = sorted({(exact_s(D[u], D[v]), v) for v in cand[u] if v != u})
        kept = nbr[u, : deg[u]].tolist()
        assert deg[u] <= R
        kept_list = []
        for s, v in order:
            if len(kept_list) == R:
                break
            occ, tight = False, False
            for w in kept_list:
                o, margin = _exact_occludes(D, u, w, v, cos_a)
                if margin != 0 and margin < 1e-12:
                    tight = True  # FP64 may round either way here
                occ = occ or o
            if tight:
                ambiguous += 1
                if v in kept:
                    kept_list.append(v)
                continue
            if occ:
                assert v not in kept
            else:
                assert v in kept
                kept_list.append(v)
        assert kept_list == kept
    assert ambiguous < 20


def test_prune_definition_on_random_shapes():
    """The same definition check over random sizes, dimensions, value ranges,
    degree bounds and angles (property test; skipped without hypothesis)."""
    pytest.importorskip("hypothesis")
    from hypothesis import given, settings, strategies as st

    @settings(max_examples=40, deadline=None)
    @given(n=st.integers(3, 50), d=st.sampled_from([4, 8, 12]), hi=st.integers(2, 9),
           R=st.integers(1, 12), alpha=st.sampled_from([60.0, 66.0, 90.0, 120.0, 180.0]),
           seed=st.integers(0, 2**31 - 1))
    def run(n, d, hi, R, alpha, seed):
        rng = np.random.default_rng(seed)
        D = rng.integers(0, hi, size=(n, d)).astype(np.float32)
        m = int(rng.integers(1, 3 * n))
        cand = rng.integers(-1, n, size=(n, m)).astype(np.int32)
        off = np.arange(n + 1, dtype=np.int64) * m
        nbr, deg = oracle.prune(D, off, cand.ravel(), R, alpha)
        cos_a = oracle.cos_alpha(alpha)
        for u in range(n):
            kept = nbr[u, :deg[u]].tolist()
            assert deg[u] <= R and len(set(kept)) == len(kept) and u not in kept
            order = sorted({(exact_s(D[u], D[v]), v) for v in cand[u] if v >= 0 and v != u})
            rebuilt = []
            for _, v in order:
                if len(rebuilt) == R:
                    break
                res = [_exact_occludes(D, u, w, v, cos_a) for w in rebuilt]
                if any(0 < mg < 1e-12 for _, mg in res):  # FP64 may round either way
                    if v in kept:
                        rebuilt.append(v)
                    continue
                if not any(o for o, _ in res):
                    rebuilt.append(v)
            assert rebuilt == kept

    run()


def test_prune_drops_self_negative_and_repeats():
    D = int_data(10, 3, 11)
    off = np.array([0, 8] + [8] * 9, np.int64)
    cand = np.array([0, -1, 3, 3, 5, -1, 0, 5], np.int32)
    nbr, deg = oracle.prune(D, off, cand, 8, 180.0)
    assert sorted(nbr[0, : deg[0]].tolist()) == [3, 5]
    assert (deg[1:] == 0).all()


def test_lemma1_probability_planar_monte_carlo():
    """Lemma 1: for a pruning triangle with angle alpha at w, a uniformly
    random query ranks w behind both u and v with probability
    (pi - alpha) / (2 pi).  Planar check with the oracle's distance."""
    rng = np.random.default_rng(12)
    for alpha in (60.0, 90.0, 120.0):
        a = math.radians(alpha)
        w = np.array([0.0, 0.0])
        u = np.array([1.0, 0.0])
        v = np.array([math.cos(a), math.sin(a)])
        nq = 20000
        Qs = rng.uniform(-400, 400, size=(nq, 2)).astype(np.float32)
        U, V, W = (p.astype(np.float32) for p in (u, v, w))
        hits = 0
        for q in Qs:
            dw = oracle.dist(q, W)
            if dw > oracle.dist(q, U) and dw > oracle.dist(q, V):
                hits += 1
        p = (math.pi - a) / (2 * math.pi)
        sigma = math.sqrt(p * (1 - p) / nq)
        assert abs(hits / nq - p) < 4 * sigma + 2e-3, alpha


# --------------------------------------------------------------------------
# reverse-edge union
# --------------------------------------------------------------------------
def test_reverse_union_is_out_plus_in_edges():
    rng = np.random.default_rng(13)
    n, R = 50, 6
    nbr = np.full((n, R), -1, np.int32)
    deg = rng.integers(0, R + 1, size=n).astype(np.int32)
    for u in range(n):
        nbr[u, : deg[u]] = rng.choice([x for x in range(n) if x != u], deg[u], replace=False)
    off, ids = oracle.reverse_union(nbr, deg)
    inn = {u: [] for u in range(n)}
    for v in range(n):
        for w in nbr[v, : deg[v]]:
            inn[int(w)].append(v)
    for u in range(n):
        row = ids[off[u]: off[u + 1]].tolist()
        assert sorted(row) == sorted(nbr[u, : deg[u]].tolist() + inn[u])


# --------------------------------------------------------------------------
# medoid and connectivity
# --------------------------------------------------------------------------
def test_medoid_is_point_nearest_exact_centroid():
    D = int_data(3000, 5, 14, hi=100)
    c = [Fraction(int(s), 3000) for s in D.astype(np.int64).sum(axis=0)]
    best = min(range(3000), key=lambda v: (sum((Fraction(int(x)) - ci) ** 2
                                               for x, ci in zip(D[v], c)), v))
    assert oracle.medoid(D) == best


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_medoid_on_real_rows_against_the_exact_centroid(seed):
    """Non-integer rows: the FP64 centroid (summed in blocks) lies within
    the summation's error bound of the exact rational centroid, and the
    medoid is the exact argmin of the rational distances whenever the gap
    between the two nearest points exceeds what that error can move."""
    rs = np.random.default_rng(40 + seed)
    n, d = 2500, 6
    D = (rs.normal(size=(n, d)) * rs.uniform(0.1, 3.0, size=d)).astype(np.float32)
    ep, c = oracle.medoid(D, return_centroid=True)
    exact = [sum(Fraction(float(x)) for x in D[:, i]) / n for i in range(d)]
    u = 2.0 ** -53
    for i in range(d):
        # n additions and one division, each relatively within u
        bound = (n + 1) * u * float(np.abs(D[:, i].astype(np.float64)).sum()) / n + 1e-300
        assert abs(Fraction(c[i]) - exact[i]) <= Fraction(bound)
    dist = sorted((sum((Fraction(float(x)) - ci) ** 2 for x, ci in zip(D[v], exact)), v)
                  for v in range(n))
    (s0, v0), (s1, _) = dist[0], dist[1]
    # the centroid's error moves each distance by at most 2 |x - c| e + e^2 per coordinate
    e = max(abs(Fraction(c[i]) - exact[i]) for i in range(d))
    spread = max(float(np.abs(D).max()), 1.0) * 2
    move = 2 * d * (2 * Fraction(spread) * e + e * e) + Fraction(8 * d * u) * s1
    assert s1 - s0 > move  # the draw is decidable
    assert ep == v0


def _reach(nbr, deg, src):
    seen = {src}
    st = [src]
    while st:
        x = st.pop()
        for y in nbr[x, : deg[x]]:
            if int(y) not in seen:
                seen.add(int(y))
                st.append(int(y))
    return seen


def test_connect_links_from_nearest_reached_node():
    rng = np.random.default_rng(15)
    A = rng.normal(0, 1, size=(20, 3))
    B = rng.normal(50, 1, size=(15, 3))
    D = np.vstack([B, A]).astype(np.float32)  # B holds ids 0..14
    n, R = 35, 4
    nbr = np.full((n, R), -1, np.int32)
    deg = np.zeros(n, np.int32)
    for u in range(n):  # a directed ring inside each group
        grp = range(0, 15) if u < 15 else range(15, 35)
        lo, hi = grp.start, grp.stop
        nbr[u, 0] = lo + (u - lo + 1) % (hi - lo)
        deg[u] = 1
    deg[16] = R
    nbr[16] = [17, 18, 19, 20]
    ep = 20
    out_nbr, out_deg, added = oracle.connect(D, nbr, deg, ep)
    assert added == 1
    assert _reach(out_nbr, out_deg, ep) == set(range(n))
    xs = D.astype(np.float64)
    cands = [x for x in range(15, 35) if deg[x] < R]
    p = min(cands, key=lambda x: (float(np.sum((xs[x] - xs[0]) ** 2)), x))
    assert out_deg[p] == deg[p] + 1 and out_nbr[p, deg[p]] == 0


def test_connect_reaches_everything_on_a_real_build():
    D, _, _ = synthetic.workload(1, n=1500, nq=1)
    ids, _ = oracle.knn(D, 10)
    off = np.arange(1501, dtype=np.int64) * 10
    nbr, deg = oracle.prune(D, off, ids.ravel(), 16, 60.0)
    ep = oracle.medoid(D)
    out_nbr, out_deg, added = oracle.connect(D, nbr, deg, ep)
    assert added > 0
    assert _reach(out_nbr, out_deg, ep) == set(range(1500))
    assert (out_deg <= 16).all()


def _connect_literal(D, nbr, deg, ep, R):
    """The connectivity reading written out with Python sets and exact
    integer distances: S = reachable from ep; while some node is unreached,
    r = the smallest unreached id, p = argmin over reached x with a free
    slot of (s(x, r), x), append r to p's list, add what r reaches to S.
    Returns (adjacency lists, added) or None when no reached node is free."""
    n = len(D)
    adj = [list(map(int, nbr[u][:deg[u]])) for u in range(n)]

    def grow(S, start):
        stack = [start]
        S.add(start)
        while stack:
            v = stack.pop()
            for w in adj[v]:
                if w >= 0 and w not in S:
                    S.add(w)
                    stack.append(w)

    S = set()
    grow(S, ep)
    added = 0
    while len(S) < n:
        r = min(set(range(n)) - S)
        free = [x for x in S if len(adj[x]) < R]
        if not free:
            return None
        p = min(free, key=lambda x: (exact_s(D[x], D[r]), x))
        adj[p].append(r)
        added += 1
        grow(S, r)
    return adj, added


@pytest.mark.parametrize("seed", range(8))
def test_connect_equals_its_literal_reading_on_random_graphs(seed):
    """Random sparse directed graphs (many components, small integer rows
    with ties): the C oracle's connectivity step adds exactly the literal
    reading's edges, or refuses exactly when it does."""
    rs = np.random.default_rng(500 + seed)
    n, R = int(rs.integers(4, 70)), int(rs.integers(1, 5))
    D = int_data(n, 3, 600 + seed, hi=6)
    nbr = np.full((n, R), -1, np.int32)
    deg = rs.integers(0, R + 1, size=n).astype(np.int32)
    deg[rs.random(n) < 0.5] = 0  # many isolated nodes
    for u in range(n):
        nbr[u, :deg[u]] = rs.choice(n, size=deg[u], replace=True)
    ep = int(rs.integers(0, n))
    want = _connect_literal(D, nbr, deg, ep, R)
    if want is None:
        assert oracle.connect(D, nbr, deg, ep)[2] < 0  # refused
        return
    adj, added = want
    out_nbr, out_deg, got_added = oracle.connect(D, nbr, deg, ep)
    assert got_added == added
    for u in range(n):
        assert out_nbr[u, :out_deg[u]].tolist() == adj[u], (seed, u)


def _connect_replace_literal(D, nbr, deg, ep, R):
    """The replacement reading written out: as _connect_literal, and when no
    reached node is free, the reached p nearest to r (by (s, id)) among
    those with an edge not added here gives its last such edge to r, then
    the reached set is recomputed from ep and r restarts from 0."""
    n = len(D)
    adj = [list(map(int, nbr[u][:deg[u]])) for u in range(n)]
    new = [[False] * len(a) for a in adj]

    def reach():
        S, stack = {ep}, [ep]
        while stack:
            v = stack.pop()
            for w in adj[v]:
                if w not in S:
                    S.add(w)
                    stack.append(w)
        return S

    S, added, rep = reach(), 0, 0
    while len(S) < n:
        r = min(set(range(n)) - S)
        key = lambda x: (exact_s(D[x], D[r]), x)
        free = [x for x in S if len(adj[x]) < R]
        if free:
            p = min(free, key=key)
            adj[p].append(r)
            new[p].append(True)
        else:
            own = [x for x in S if not all(new[x])]
            if not own:
                return None
            p = min(own, key=key)
            j = max(i for i, f in enumerate(new[p]) if not f)
            adj[p][j], new[p][j] = r, True
            rep += 1
        added += 1
        S = reach()
    return adj, added, rep


@pytest.mark.parametrize("seed", range(10))
def test_connect_replacement_equals_its_literal_reading(seed):
    """The edge-replacement reading (for graphs whose reached nodes are all
    full) equals its literal restatement, reaches every node and keeps every
    degree within R, on random graphs where the plain step often refuses."""
    rs = np.random.default_rng(700 + seed)
    n, R = int(rs.integers(4, 50)), int(rs.integers(1, 4))
    D = int_data(n, 3, 800 + seed, hi=6)
    nbr = np.full((n, R), -1, np.int32)
    deg = np.full(n, R, np.int32)  # full rows: the plain step mostly refuses
    deg[rs.random(n) < 0.2] = 0
    for u in range(n):
        nbr[u, :deg[u]] = rs.choice(n, size=deg[u], replace=True)
    ep = int(rs.integers(0, n))
    want = _connect_replace_literal(D, nbr, deg, ep, R)
    out_nbr, out_deg, added, rep = oracle.connect_replace(D, nbr, deg, ep)
    if want is None:
        assert added < 0
        return
    adj, w_added, w_rep = want
    assert (added, rep) == (w_added, w_rep)
    for u in range(n):
        assert out_nbr[u, :out_deg[u]].tolist() == adj[u], (seed, u)
    assert (out_deg <= R).all()
    assert _reach(out_nbr, out_deg, ep) == set(range(n))


def test_connect_replacement_links_full_tight_clusters():
    """Tight clusters whose pruned rows are all full (the situation of the
    4,096-cluster 384-d recipe at alpha 66): the plain step refuses, the
    replacement reading connects everything within R."""
    rs = np.random.default_rng(41)
    centres = rs.normal(0, 10, (12, 64))
    D = np.vstack([c + rs.normal(0, 0.05, (16, 64)) for c in centres]).astype(np.float32)
    n, K, R = D.shape[0], 8, 4
    ids, _ = oracle.knn(D, K)
    nbr, deg = oracle.prune(D, np.arange(n + 1, dtype=np.int64) * K, ids.ravel(), R, 66.0)
    ep = oracle.medoid(D)
    reach0 = _reach(nbr, deg, ep)
    assert len(reach0) < n and all(deg[x] == R for x in reach0)
    assert oracle.connect(D, nbr, deg, ep)[2] < 0
    out_nbr, out_deg, added, rep = oracle.connect_replace(D, nbr, deg, ep)
    assert added > 0 and rep > 0
    assert _reach(out_nbr, out_deg, ep) == set(range(n)) and (out_deg <= R).all()


# --------------------------------------------------------------------------
# beam search
# --------------------------------------------------------------------------
def test_search_on_complete_graph_is_exact_knn():
    D = int_data(40, 4, 16, hi=9)
    Q = int_data(6, 4, 17, hi=9)
    n = 40
    nbr = np.array([[v for v in range(n) if v != u] for u in range(n)], np.int32)
    deg = np.full(n, n - 1, np.int32)
    ids, ds = oracle.search(D, nbr, deg, Q, 3, 7, n)
    for q in range(6):
        pairs = sorted((exact_s(Q[q], D[v]), v) for v in range(n))[:7]
        assert ids[q].tolist() == [v for _, v in pairs]


def test_search_recall_grows_with_the_pool_width():
    """A wider pool explores a superset of the routes of a narrower one, so
    recall@10 on a pruned graph rises with L (soft: a small dip is allowed,
    the trend is not)."""
    D, Q, _ = synthetic.workload(1, n=3000, nq=60)
    nbr, deg, ep = oracle.build_rng(D, 16, 48, 12, 66.0, 60.0, 1)  # connected
    gt = oracle.knn(D, 10, Q=Q)
    rec = []
    for L in (10, 20, 40, 80, 160):
        found, _ = oracle.search(D, nbr, deg, Q, ep, 10, L)
        rec.append(oracle.recall_at_k(found, Q, D, 10, gt=gt))
    assert all(b >= a - 0.02 for a, b in zip(rec, rec[1:]))
    assert rec[-1] > rec[0]


def test_search_on_path_graph_walks_to_the_target():
    n = 60
    D = np.arange(n, dtype=np.float32).reshape(n, 1)
    nbr = np.full((n, 2), -1, np.int32)
    deg = np.zeros(n, np.int32)
    for u in range(n):
        row = [x for x in (u - 1, u + 1) if 0 <= x < n]
        nbr[u, : len(row)] = row
        deg[u] = len(row)
    Q = np.array([[41.2], [3.9], [58.6]], np.float32)
    ids, ds, ne = oracle.search(D, nbr, deg, Q, 0, 2, 2, return_expanded=True)
    assert ids.tolist() == [[41, 42], [4, 3], [59, 58]]


def test_search_visited_policy_does_not_change_the_pool():
    D, Q, _ = synthetic.workload(1, n=1200, nq=40)
    ids, _ = oracle.knn(D, 8)
    off = np.arange(1201, dtype=np.int64) * 8
    nbr, deg = oracle.prune(D, off, ids.ravel(), 8, 70.0)
    starts = np.random.default_rng(18).integers(0, 1200, size=40)
    for L in (4, 17, 50):
        a = oracle.search(D, nbr, deg, Q, starts, L, L, policy=0)
        b = oracle.search(D, nbr, deg, Q, starts, L, L, policy=1)
        assert (a[0] == b[0]).all() and (a[1] == b[1]).all()


def _kann_search_literal(D, nbr, deg, q, starts, k, L):
    """Algorithm 1 written out with Python containers and exact integer
    distances: the pool holds (s, id) pairs sorted ascending and cut to L;
    the first entry not yet expanded is expanded next; a node is evaluated
    once (visited set) and an evicted node never comes back."""
    pool = sorted((exact_s(q, D[e]), int(e)) for e in starts)[:L]
    visited = {int(e) for e in starts}
    expanded = set()
    while True:
        nxt = next((v for _, v in pool if v not in expanded), None)
        if nxt is None:
            break
        expanded.add(nxt)
        for w in nbr[nxt][:deg[nxt]]:
            w = int(w)
            if w < 0 or w in visited:
                continue
            visited.add(w)
            pool.append((exact_s(q, D[w]), w))
        pool = sorted(pool)[:L]
    out = [v for _, v in pool[:k]]
    return out + [-1] * (k - len(out))


@pytest.mark.parametrize("seed", range(6))
def test_search_equals_a_literal_algorithm1_on_random_graphs(seed):
    """Tiny random directed graphs (uneven degrees, -1 padding, many exact
    ties from small integer values), one or several entry points, random
    k <= L: the C oracle's search returns the literal restatement's lists."""
    rs = np.random.default_rng(100 + seed)
    n, d, R = int(rs.integers(5, 60)), int(rs.integers(1, 5)), int(rs.integers(1, 7))
    D = int_data(n, d, 200 + seed, hi=5)
    nq = 12
    Q = int_data(nq, d, 300 + seed, hi=5)
    nbr = np.full((n, R), -1, np.int32)
    deg = rs.integers(0, R + 1, size=n).astype(np.int32)
    for u in range(n):
        nbr[u, :deg[u]] = rs.choice(n, size=deg[u], replace=True)
    width = int(rs.integers(1, 4))
    starts = np.array([rs.choice(n, size=min(width, n), replace=False) for _ in range(nq)],
                      np.int32)
    L = int(rs.integers(1, 12))
    k = int(rs.integers(1, L + 1))
    ids, ds = oracle.search(D, nbr, deg, Q, starts, k, L)
    for i in range(nq):
        want = _kann_search_literal(D, nbr, deg, Q[i], starts[i], k, L)
        assert ids[i].tolist() == want, (seed, i)
        got = [exact_s(Q[i], D[v]) for v in want if v >= 0]
        assert ds[i][:len(got)].tolist() == got


def _path_layer(members, edges, R):
    """An oracle.Layer over the ascending ids `members` with the undirected
    `edges` (pairs of point ids), adjacency rows in member order."""
    members = sorted(members)
    row = {v: i for i, v in enumerate(members)}
    nbr = np.full((len(members), R), -1, np.int32)
    deg = np.zeros(len(members), np.int32)
    for a, b in edges:
        for x, y in ((a, b), (b, a)):
            nbr[row[x], deg[row[x]]] = y
            deg[row[x]] += 1
    return oracle.Layer(np.array(members, np.int32), nbr, deg, R)


def test_search_nswg_hand_built_descent():
    """Points 0..39 on a line.  Layer 0 is two paths, 0-...-19 and
    20-...-39, so a search that starts on the wrong side can never cross;
    layer 1 holds {0, 10, 30} linked 0-10-30; layer 2 holds {0}.  Greedy
    routing from ep 0 for the query 33.2 goes 0 -> 10 -> 30 on layer 1, and
    the width-4 search of layer 0 from 30 returns 33, 34, 32.  For 7.4 it
    stops at 10 and returns 7, 8, 6.  Skipping layer 1, or reading layer 1's
    rows through the wrong map, starts layer 0 at 0 and cannot reach 33."""
    n = 40
    D = np.arange(n, dtype=np.float32).reshape(n, 1)
    base_edges = [(u, u + 1) for u in range(19)] + [(u, u + 1) for u in range(20, 39)]
    base = _path_layer(range(n), base_edges, 2)
    base.gid = None
    lay1 = _path_layer([0, 10, 30], [(0, 10), (10, 30)], 2)
    lay2 = _path_layer([0], [], 1)
    Q = np.array([[33.2], [7.4]], np.float32)
    ids, _ = oracle.search_nswg(D, [base, lay1, lay2], 0, Q, 3, 4, "l2")
    assert ids.tolist() == [[33, 34, 32], [7, 8, 6]]
    # without the routing layer the base search from 0 stays on 0..19
    ids, _ = oracle.search_nswg(D, [base, lay2], 0, Q, 3, 4, "l2")
    assert ids.tolist() == [[19, 18, 17], [7, 8, 6]]


def _layered_search_literal(D, layers, ep, q, k, ef, ef_upper):
    """The layered query written out: w <- ep; for each layer from the top
    down to layer 1, w <- the nearest result of Algorithm 1 on that layer
    (pool ef_upper, from w); then Algorithm 1 on layer 0 (pool ef, from w).
    Adjacency is looked up by point id in a dictionary per layer."""
    w = ep
    for i in range(len(layers) - 1, -1, -1):
        lay = layers[i]
        gid = range(lay.nbr.shape[0]) if lay.gid is None else lay.gid.tolist()
        adj = {int(v): [int(x) for x in lay.nbr[r][:lay.deg[r]]] for r, v in enumerate(gid)}
        L = ef if i == 0 else ef_upper
        pool = [(exact_s(q, D[w]), w)]
        visited, expanded = {w}, set()
        while True:
            nxt = next((v for _, v in pool if v not in expanded), None)
            if nxt is None:
                break
            expanded.add(nxt)
            for x in adj[nxt]:
                if x not in visited:
                    visited.add(x)
                    pool.append((exact_s(q, D[x]), x))
            pool = sorted(pool)[:L]
        if i > 0:
            w = pool[0][1]
        else:
            out = [v for _, v in pool[:k]]
            return out + [-1] * (k - len(out))


@pytest.mark.parametrize("seed", range(6))
def test_search_nswg_equals_a_literal_layered_descent(seed):
    """Random nested layers (each a subset of the one below, uneven random
    adjacency among its members, exact integer distances with many ties),
    random ef_upper: oracle.search_nswg returns the literal descent's lists."""
    rs = np.random.default_rng(700 + seed)
    n, d = int(rs.integers(20, 80)), int(rs.integers(1, 4))
    D = int_data(n, d, 710 + seed, hi=6)
    nq = 10
    Q = int_data(nq, d, 720 + seed, hi=6)
    members = list(range(n))
    layers = []
    for i in range(int(rs.integers(2, 5))):
        if i > 0:
            keep = max(1, len(members) // int(rs.integers(2, 5)))
            members = sorted(rs.choice(members, size=keep, replace=False).tolist())
        R = int(rs.integers(1, 6))
        m = len(members)
        nbr = np.full((m, R), -1, np.int32)
        deg = rs.integers(0, R + 1, size=m).astype(np.int32)
        for r in range(m):
            nbr[r, :deg[r]] = rs.choice(members, size=deg[r], replace=True)
        gid = None if i == 0 else np.array(members, np.int32)
        layers.append(oracle.Layer(gid, nbr, deg, R))
    ep = members[0]
    ef = int(rs.integers(1, 10))
    k = int(rs.integers(1, ef + 1))
    ef_upper = int(rs.integers(1, 4))
    ids, _ = oracle.search_nswg(D, layers, ep, Q, k, ef, "l2", ef_upper=ef_upper)
    for i in range(nq):
        want = _layered_search_literal(D, layers, ep, Q[i], k, ef, ef_upper)
        assert ids[i].tolist() == want, (seed, i)


def test_acquire_on_complete_graph_is_exact_knn_minus_self():
    D = int_data(30, 3, 19, hi=7)
    n = 30
    nbr = np.array([[v for v in range(n) if v != u] for u in range(n)], np.int32)
    deg = np.full(n, n - 1, np.int32)
    cand = oracle.acquire(D, nbr, deg, 12)
    ids, _ = oracle.knn(D, 11)
    assert (cand[:, :11] == ids).all() and (cand[:, 11] == -1).all()


# --------------------------------------------------------------------------
# IterNSG composition and the hierarchical build
# --------------------------------------------------------------------------
def test_build_rng_equals_composed_steps():
    D, _, _ = synthetic.workload(1, n=800, nq=1)
    K, L, R = 10, 24, 12
    nbr, deg, ep = oracle.build_rng(D, K, L, R, 66.0, 60.0, iters=1)
    ids, _ = oracle.knn(D, K)
    assert ep == oracle.medoid(D)

    def refine(off, cand, alpha, do_connect):
        n1, d1 = oracle.prune(D, off, cand, R, alpha)
        uo, ui = oracle.reverse_union(n1, d1)
        n2, d2 = oracle.prune(D, uo, ui, R, alpha)
        if do_connect:
            n2, d2, _ = oracle.connect(D, n2, d2, ep)
        return n2, d2

    g, gd = refine(np.arange(801, dtype=np.int64) * K, ids.ravel(), 66.0, True)
    cand = oracle.acquire(D, g, gd, L)
    g2, gd2 = refine(np.arange(801, dtype=np.int64) * L, cand.ravel(), 60.0, True)
    assert (g2 == nbr).all() and (gd2 == deg).all()
    assert _reach(nbr, deg, ep) == set(range(800))


def test_splitmix64_published_outputs():
    for state, out in _read_golden("splitmix64_seed0.txt"):
        assert oracle.splitmix64(int(state, 16)) == int(out, 16)


def test_levels_follow_the_geometric_law():
    n, M = 200_000, 16
    lev = oracle.levels(n, 99, M)
    for i in (1, 2, 3):
        p = M ** (-i)
        frac = float((lev >= i).mean())
        assert abs(frac - p) < 5 * math.sqrt(p * (1 - p) / n), i


def test_nswg_small_layers_are_complete_and_nested():
    D = synthetic.unit_gaussian(900, 8, 20)
    layers, ep, lev = oracle.build_nswg(D, 10, 20, 4, 8, iters=1, seed=3)
    assert len(layers) == int(lev.max()) + 1
    for i, lay in enumerate(layers):
        assert (lay.gid == np.nonzero(lev >= i)[0]).all()
        if i > 0:
            assert set(lay.gid.tolist()) <= set(layers[i - 1].gid.tolist())
        m = lay.gid.shape[0]
        if m <= lay.R:
            for a in range(m):
                assert sorted(lay.nbr[a, : lay.deg[a]].tolist()) == sorted(
                    int(x) for x in lay.gid if x != lay.gid[a])
        assert (lay.deg <= lay.R).all()
    assert ep == int(layers[-1].gid[0])


def test_recall_helper_on_hand_made_lists():
    D = np.array([[0.0], [1.0], [2.0], [2.0], [5.0]], np.float32)
    Q = np.array([[0.0]], np.float32)
    gt = oracle.knn(D, 3, Q=Q)
    # the 3rd distance is a tie between ids 2 and 3: either counts
    assert oracle.recall_at_k(np.array([[0, 1, 3]]), Q, D, 3, gt=gt) == 1.0
    assert oracle.recall_at_k(np.array([[0, 0, 4]]), Q, D, 3, gt=gt) == pytest.approx(1 / 3)
    assert oracle.recall_at_k(np.array([[-1, 2, 1]]), Q, D, 3, gt=gt) == pytest.approx(2 / 3)


# ------------------------------------------------------------- insertion
def _rng_set(P, u, others):
    """RNG pruning of u's candidates `others` written out in exact integers:
    scan by (s(u, v), v) and keep v unless a kept w is strictly closer to u
    and strictly closer to v than u is to v (Algorithm 3 at alpha = 60)."""
    def s(a, b):
        return int(((P[a].astype(np.int64) - P[b].astype(np.int64)) ** 2).sum())
    kept = []
    for v in sorted(others, key=lambda v: (s(u, v), v)):
        if not any(s(u, w) < s(u, v) and s(v, w) < s(u, v) for w in kept):
            kept.append(v)
    return set(kept)


def test_insert_into_complete_layer_links_the_rng_neighbours():
    """An exhaustive search (ef >= n on a complete layer) makes N(u) the RNG
    set of u over all points, and every linked v's list the RNG set of v
    over its old list plus u."""
    rng = np.random.default_rng(11)
    P = rng.integers(0, 60, size=(31, 2)).astype(np.float32)
    P = np.concatenate([P, np.zeros((31, 2), np.float32)], axis=1)  # d = 4
    n_old = 30
    layers, ep, _ = oracle.build_nswg(P[:n_old], 8, 40, 16, 32, 60.0, 60.0, 1, "l2", 3,
                                      lev=np.zeros(n_old, np.int32))
    assert len(layers) == 1 and (layers[0].deg == n_old - 1).all()  # complete
    new = oracle.insert_batch(P, layers, ep, n_old, 40, 60.0, "l2", 3, 16)
    L0 = new[0]
    u = n_old
    got = set(L0.nbr[u, :L0.deg[u]].tolist())
    assert got == _rng_set(P, u, list(range(n_old)))
    for v in range(n_old):
        lst = set(L0.nbr[v, :L0.deg[v]].tolist())
        if v in got:
            assert lst == _rng_set(P, v, [w for w in range(n_old + 1) if w != v])
        else:
            assert lst == set(layers[0].nbr[v, :layers[0].deg[v]].tolist())


def test_insert_levels_follow_the_build_draw_capped_at_the_top():
    D, _, _ = synthetic.workload(1, n=900, nq=1)
    layers, ep, lev = oracle.build_nswg(D[:800], 16, 32, 16, 32, 70.0, 60.0, 1, "l2", 9)
    new = oracle.insert_batch(D, layers, ep, 800, 32, 60.0, "l2", 9, 16)
    top = len(layers) - 1
    want = np.minimum(oracle.levels(900, 9, 16)[800:], top)
    for i, L in enumerate(new):
        members = set(L.gid.tolist())
        assert set(layers[i].gid.tolist()) <= members
        assert {800 + k for k in np.nonzero(want >= i)[0]} == members - set(layers[i].gid.tolist())
        assert (L.deg <= L.R).all() and (np.diff(L.gid) > 0).all()
    assert (new[0].deg[800:] > 0).all()


# --------------------------------------------------------------------------
# qualitative claims of the paper (soft trends)
# --------------------------------------------------------------------------
def test_more_iterations_do_not_lower_recall():
    """Exp. 1-a: further OptKCNA iterations improve the graph, with little
    change after the second (soft: non-decreasing recall at a fixed beam)."""
    D, Q, _ = synthetic.workload(1, n=2000, nq=80)
    gt = oracle.knn(D, 10, Q=Q)
    rec = []
    for it in (0, 1, 2):
        nbr, deg, ep = oracle.build_rng(D, 16, 48, 16, 66.0, 60.0, it)
        ids, _ = oracle.search(D, nbr, deg, Q, ep, 10, 24)
        rec.append(oracle.recall_at_k(ids, Q, D, 10, gt=gt))
    assert rec[1] >= rec[0] and rec[2] >= rec[1] - 0.01, rec


def test_wider_alpha_loses_less_kcna_quality():
    """Section 4.2 (Lemma 1, Theorem 2): pruning with a larger alpha loses
    less k-CNA quality; alpha = 60 (RNG pruning) keeps the fewest edges."""
    D, _, _ = synthetic.workload(1, n=2000, nq=1)
    ids, _ = oracle.knn(D, 16)
    off = np.arange(2001, dtype=np.int64) * 16
    ep = oracle.medoid(D)
    quality, degree = [], []
    for a in (60.0, 66.0, 90.0):
        N, dg = oracle.prune(D, off, ids.ravel(), 16, a)
        uoff, uids = oracle.reverse_union(N, dg)
        G, gd = oracle.prune(D, uoff, uids, 16, a)
        G, gd, _ = oracle.connect(D, G, gd, ep)
        C = oracle.acquire(D, G, gd, 32)
        quality.append(oracle.kcna_recall(D, C, 10).mean())
        degree.append(gd.mean())
    assert quality[0] <= quality[1] <= quality[2], quality
    assert degree[0] < degree[1] <= degree[2], degree

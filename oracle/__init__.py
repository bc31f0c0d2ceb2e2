"""FP64 CPU oracle for the graph-construction path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and
shares no code with it.  The arithmetic lives in ``oracle.c``; this module
compiles it (gcc, ``-ffp-contract=off``), marshals numpy arrays and composes
the hierarchical build of Algorithm 7 from the C pieces.  The FP8 row format
of the screened queries (not a subject of the paper) is written out here in
Python from the definition of the number format.

Every function of the method names the passage of arXiv 2410.01231 it
restates.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

METRICS = {"l2": 0, "cosine": 1, "ip": 2}

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _get():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        P = C.c_void_p
        i64, i32, dbl = C.c_int64, C.c_int, C.c_double
        lib.or_dist.restype = dbl
        lib.or_dist.argtypes = [P, P, i32, i32]
        lib.or_knn.restype = i32
        lib.or_knn.argtypes = [P, i64, i32, i32, P, i64, P, i32, P, P]
        lib.or_prune.restype = i32
        lib.or_prune.argtypes = [P, i64, i32, i32, P, P, i32, dbl, i32, P, P]
        lib.or_reverse_union.restype = i64
        lib.or_reverse_union.argtypes = [P, P, i64, i32, P, P]
        lib.or_medoid.restype = i64
        lib.or_medoid.argtypes = [P, i64, i32, i32, P]
        lib.or_connect.restype = i64
        lib.or_connect.argtypes = [P, i64, i32, i32, P, P, i32, i64]
        lib.or_connect_replace.restype = i64
        lib.or_connect_replace.argtypes = [P, i64, i32, i32, P, P, i32, i64, P]
        lib.or_search.restype = i32
        lib.or_search.argtypes = [P, i64, i32, i32, P, P, i32, P, P, i64, P, i32, i32, i32,
                                  i32, P, P, P]
        lib.or_knn_descent.restype = i32
        lib.or_knn_descent.argtypes = [P, i64, i32, i32, i32, i32, P, P, P]
        lib.or_acquire.restype = i32
        lib.or_acquire.argtypes = [P, i64, i32, i32, P, P, i32, i32, P, P]
        lib.or_build_rng.restype = i64
        lib.or_build_rng.argtypes = [P, i64, i32, i32, i32, i32, i32, dbl, i32, dbl, i32, i32,
                                     i32, P, P]
        lib.or_levels.restype = None
        lib.or_levels.argtypes = [i64, C.c_uint64, i32, P]
        lib.or_splitmix64.restype = C.c_uint64
        lib.or_splitmix64.argtypes = [C.c_uint64]
        lib.or_num_threads.restype = i32
        lib.or_set_threads.argtypes = [i32]
        _lib = lib
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(D):
    return np.ascontiguousarray(D, dtype=np.float32)


def num_threads() -> int:
    return _get().or_num_threads()


def set_threads(t: int) -> None:
    _get().or_set_threads(int(t))


def cos_alpha(alpha_deg: float) -> float:
    """cos(alpha) for the angle clause of alpha-pruning (Section 4.1)."""
    return math.cos(alpha_deg * math.pi / 180.0)


# --------------------------------------------------------------------------
def dist(x: np.ndarray, y: np.ndarray, metric: str = "l2") -> float:
    """s(x, y) in FP64 (Section 2; squared chord for unit-norm metrics)."""
    x, y = _f32(x), _f32(y)
    return _get().or_dist(_p(x), _p(y), x.shape[0], METRICS[metric])


def knn(D, K: int, metric: str = "l2", Q=None, rows=None):
    """Exact K nearest neighbours by (s, id); self excluded when Q is None.
    With ``rows`` only those points' rows of the graph are computed."""
    D = _f32(D)
    n, d = D.shape
    if rows is not None:
        rows = np.ascontiguousarray(rows, np.int64)
        Qa, excl = np.ascontiguousarray(D[rows]), rows
    elif Q is None:
        Qa, excl = D, np.arange(n, dtype=np.int64)
    else:
        Qa, excl = _f32(Q), None
    nq = Qa.shape[0]
    ids = np.empty((nq, K), np.int32)
    ds = np.empty((nq, K), np.float64)
    rc = _get().or_knn(_p(D), n, d, METRICS[metric], _p(Qa), nq, _p(excl), K, _p(ids), _p(ds))
    assert rc == 0
    return ids, ds


def prune(D, off, cand, R: int, alpha_deg: float, metric: str = "l2"):
    """alpha-pruning of every CSR row (Section 4.1 rule, Algorithm 3 scan)."""
    D = _f32(D)
    n, d = D.shape
    off = np.ascontiguousarray(off, np.int64)
    cand = np.ascontiguousarray(cand, np.int32)
    nbr = np.empty((n, R), np.int32)
    deg = np.empty(n, np.int32)
    rc = _get().or_prune(_p(D), n, d, METRICS[metric], _p(off), _p(cand), R,
                         cos_alpha(alpha_deg), int(alpha_deg == 60.0), _p(nbr), _p(deg))
    assert rc == 0
    return nbr, deg


def knn_descent(D, init, iters: int, metric: str = "l2"):
    """kNN graph refined by 2-hop neighbours (the KGraph iteration as Exp. 12
    describes it): N_0(u) = the ids of init[u] sorted by (s, id); each
    iteration N(u) <- the K best by (s, id) of N(u) and the lists of its
    members, u excluded.  Returns (ids [n][K], dist [n][K] FP64)."""
    D = _f32(D)
    n, d = D.shape
    init = np.ascontiguousarray(init, np.int32)
    K = init.shape[1]
    ids = np.empty((n, K), np.int32)
    dist = np.empty((n, K), np.float64)
    rc = _get().or_knn_descent(_p(D), n, d, METRICS[metric], K, int(iters), _p(init), _p(ids),
                               _p(dist))
    assert rc == 0
    return ids, dist


def reverse_union(nbr, deg):
    """Row u = N(u) then {v : u in N(v)} (Algorithm 2)."""
    nbr = np.ascontiguousarray(nbr, np.int32)
    deg = np.ascontiguousarray(deg, np.int32)
    n, R = nbr.shape
    off = np.empty(n + 1, np.int64)
    tot = _get().or_reverse_union(_p(nbr), _p(deg), n, R, _p(off), None)
    ids = np.empty(max(tot, 1), np.int32)
    _get().or_reverse_union(_p(nbr), _p(deg), n, R, _p(off), _p(ids))
    return off, ids[:tot]


def medoid(D, metric: str = "l2", return_centroid: bool = False):
    """Point nearest the centroid (Section 3.1, search phase); with
    return_centroid also the FP64 centroid it used."""
    D = _f32(D)
    c = np.zeros(D.shape[1], np.float64)
    ep = int(_get().or_medoid(_p(D), D.shape[0], D.shape[1], METRICS[metric], _p(c)))
    return (ep, c) if return_centroid else ep


def connect(D, nbr, deg, ep: int, metric: str = "l2"):
    """Link unreachable components (Algorithm 2); returns copies."""
    D = _f32(D)
    nbr = np.array(nbr, np.int32, copy=True)
    deg = np.array(deg, np.int32, copy=True)
    n, R = nbr.shape
    added = _get().or_connect(_p(D), n, D.shape[1], METRICS[metric], _p(nbr), _p(deg), R, ep)
    return nbr, deg, int(added)


def connect_replace(D, nbr, deg, ep: int, metric: str = "l2"):
    """The connectivity step with edge replacement (a reading for graphs whose
    reached nodes are all full; the builds use ``connect``): when no reached
    node has a free slot, the nearest reached node with an original edge
    gives up its last one for the unreached node, and reachability is
    recomputed.  Returns copies and (edges added, of which replacements);
    edges added is negative when nothing can be linked."""
    D = _f32(D)
    nbr = np.array(nbr, np.int32, copy=True)
    deg = np.array(deg, np.int32, copy=True)
    n, R = nbr.shape
    rep = np.zeros(1, np.int64)
    added = _get().or_connect_replace(_p(D), n, D.shape[1], METRICS[metric], _p(nbr), _p(deg),
                                      R, ep, _p(rep))
    return nbr, deg, int(added), int(rep[0])


def search(D, nbr, deg, Q, starts, k: int, L: int, metric: str = "l2", rows=None,
           policy: int = 0, return_expanded: bool = False):
    """KANNSearch (Algorithm 1) for every query row.

    ``starts`` is an int, a 1-D array (one entry point per query) or a 2-D
    array (several per query).
    """
    D = _f32(D)
    Q = _f32(Q)
    nbr = np.ascontiguousarray(nbr, np.int32)
    deg = np.ascontiguousarray(deg, np.int32)
    n, d = D.shape
    nq = Q.shape[0]
    st = np.asarray(starts, dtype=np.int32)
    if st.ndim == 0:
        st = np.full((nq, 1), int(st), np.int32)
    elif st.ndim == 1:
        st = st.reshape(nq, 1)
    st = np.ascontiguousarray(st)
    rows_a = None if rows is None else np.ascontiguousarray(rows, np.int32)
    ids = np.empty((nq, k), np.int32)
    ds = np.empty((nq, k), np.float64)
    ne = np.zeros(1, np.int64)
    rc = _get().or_search(_p(D), n, d, METRICS[metric], _p(nbr), _p(deg), nbr.shape[1],
                          _p(rows_a), _p(Q), nq, _p(st), st.shape[1], k, L, policy, _p(ids),
                          _p(ds), _p(ne))
    assert rc == 0
    if return_expanded:
        return ids, ds, int(ne[0])
    return ids, ds


def acquire(D, nbr, deg, L: int, metric: str = "l2"):
    """C(u) <- KANNSearch(G, u, L, L, u) minus u (Algorithm 5)."""
    D = _f32(D)
    nbr = np.ascontiguousarray(nbr, np.int32)
    deg = np.ascontiguousarray(deg, np.int32)
    n, d = D.shape
    cand = np.empty((n, L), np.int32)
    rc = _get().or_acquire(_p(D), n, d, METRICS[metric], _p(nbr), _p(deg), nbr.shape[1], L,
                           _p(cand), None)
    assert rc == 0
    return cand


def build_rng(D, K: int, L: int, R: int, alpha_deg: float = 66.0, alpha_final_deg: float = 60.0,
              iters: int = 2, metric: str = "l2", connect_final: bool = True):
    """IterNSG with fixed I (Algorithm 6 + Algorithm 5); returns (nbr, deg, ep)."""
    D = _f32(D)
    n, d = D.shape
    nbr = np.empty((n, R), np.int32)
    deg = np.empty(n, np.int32)
    ep = _get().or_build_rng(_p(D), n, d, METRICS[metric], K, L, R, cos_alpha(alpha_deg),
                             int(alpha_deg == 60.0), cos_alpha(alpha_final_deg),
                             int(alpha_final_deg == 60.0), iters, int(connect_final),
                             _p(nbr), _p(deg))
    if ep < 0:
        raise RuntimeError(f"oracle build_rng failed ({ep})")
    return nbr, deg, int(ep)


def splitmix64(x: int) -> int:
    """One SplitMix64 output for state x (the generator behind the levels)."""
    return int(_get().or_splitmix64(x))


def levels(n: int, seed: int, M: int) -> np.ndarray:
    """HNSW levels floor(-ln U / ln M), U from SplitMix64 (Algorithm 7)."""
    out = np.empty(n, np.int32)
    _get().or_levels(n, seed, M, _p(out))
    return out


# --------------------------------------------------------------------------
# Hierarchical (NSWG) build, Algorithm 7, and its layered query.
# --------------------------------------------------------------------------
class Layer:
    __slots__ = ("gid", "nbr", "deg", "R")

    def __init__(self, gid, nbr, deg, R):
        self.gid, self.nbr, self.deg, self.R = gid, nbr, deg, R


def build_nswg(D, K: int, L: int, M: int, R0: int, alpha_deg: float = 66.0,
               alpha_final_deg: float = 60.0, iters: int = 2, metric: str = "cosine",
               seed: int = 0, lev=None):
    """OptHNSW (Algorithm 7).

    Levels are drawn for every point up front; layer i holds
    D_i = {u : l(u) >= i} (ascending ids).  A layer with |D_i| <= M_i is a
    complete graph (every other member, by (s, id)); any other layer is the
    IterNSG build of D_i with pool width ef = L, whose final refinement
    skips the connectivity step (Section 5.3).  M_0 = R0 and M_i = M for
    i >= 1.  ep is the smallest id on the top layer (a deterministic reading
    of the paper's random choice of the entry).  Layer adjacency holds global ids.
    """
    D = _f32(D)
    n = D.shape[0]
    lev = levels(n, seed, M) if lev is None else np.asarray(lev, np.int32)
    top = int(lev.max())
    layers = []
    for i in range(top + 1):
        gid = np.nonzero(lev >= i)[0].astype(np.int32)
        Ri = R0 if i == 0 else M
        m = gid.shape[0]
        Di = D[gid]
        if m <= Ri:
            nbr = np.full((m, Ri), -1, np.int32)
            deg = np.zeros(m, np.int32)
            for a in range(m):
                others = [(dist(Di[a], Di[b], metric), int(gid[b])) for b in range(m) if b != a]
                others.sort()
                for j, (_, g) in enumerate(others):
                    nbr[a, j] = g
                deg[a] = len(others)
        else:
            lnbr, deg, _ = build_rng(Di, K, L, Ri, alpha_deg, alpha_final_deg, iters, metric,
                                     connect_final=False)
            nbr = np.where(lnbr >= 0, gid[np.maximum(lnbr, 0)], -1).astype(np.int32)
        layers.append(Layer(gid, nbr, deg, Ri))
    ep = int(layers[top].gid[0])
    return layers, ep, lev


def search_nswg(D, layers, ep: int, Q, k: int, ef: int, metric: str = "cosine",
                ef_upper: int = 1):
    """Layered query: w <- first of KANNSearch(G_i, q, 1, ef_upper, w) from
    the top layer down to layer 1, then KANNSearch(G_0, q, k, ef, w)
    (pattern of Algorithm 4; ef_upper = 1 is greedy routing)."""
    D = _f32(D)
    Q = _f32(Q)
    n = D.shape[0]
    nq = Q.shape[0]
    w = np.full(nq, ep, np.int32)
    for i in range(len(layers) - 1, 0, -1):
        lay = layers[i]
        rows = np.full(n, -1, np.int32)
        rows[lay.gid] = np.arange(lay.gid.shape[0], dtype=np.int32)
        ids, _ = search(D, lay.nbr, lay.deg, Q, w, 1, ef_upper, metric, rows=rows)
        w = ids[:, 0].copy()
    base = layers[0]
    return search(D, base.nbr, base.deg, Q, w, k, ef, metric)


def insert_batch(D_all, layers, ep: int, n_old: int, ef: int, alpha_deg: float = 60.0,
                 metric: str = "l2", seed: int = 0, M: int = 16, ef_upper: int = 1):
    """Batched insertion of the points n_old..len(D_all)-1 into a layered
    index, every new point against the graph as it was before the batch.

    Per new point u (the search and refinement phases of Algorithm 4):
    its level l(u) is the SplitMix64 draw of the build (Algorithm 7)
    capped at the top layer; w <- ep, then w <- first of
    KANNSearch(G_i, u, 1, ef_upper, w) for the layers above l(u); for
    i = l(u)..0: W_i <- KANNSearch(G_i, u, ef, ef, w), w <- W_i[0], and
    N_i(u) <- Prune(u, W_i, R_i, alpha).  Then every old v with new
    in-edges I_i(v) = {u : v in N_i(u)} gets
    N_i(v) <- Prune(v, N_i(v) | I_i(v), R_i, alpha) from its list before
    the batch (the reverse-edge step of Algorithm 4).  New nodes are
    appended to the layers in id order.  Returns new Layer objects.
    """
    D_all = _f32(D_all)
    N = D_all.shape[0]
    m = N - n_old
    top = len(layers) - 1
    lev = np.minimum(levels(N, seed, M)[n_old:], top)
    Q = D_all[n_old:]
    w = np.full(m, ep, np.int32)
    out = [None] * (top + 1)
    for i in range(top, -1, -1):
        lay = layers[i]
        Ri = lay.R
        rows = None
        if i > 0:
            rows = np.full(N, -1, np.int32)
            rows[lay.gid] = np.arange(lay.gid.shape[0], dtype=np.int32)
        S = np.nonzero(lev >= i)[0]
        B = np.nonzero(lev < i)[0]
        if i >= 1 and B.shape[0]:
            ids, _ = search(D_all, lay.nbr, lay.deg, Q[B], w[B], 1, ef_upper, metric, rows=rows)
            w[B] = ids[:, 0]
        gid = lay.gid.copy()
        nbr = lay.nbr.copy()
        deg = lay.deg.copy()
        if S.shape[0]:
            W, _ = search(D_all, lay.nbr, lay.deg, Q[S], w[S], ef, ef, metric, rows=rows)
            w[S] = W[:, 0]
            # N_i(u) for the new points: rows of a CSR over all N points
            cnt = np.zeros(N, np.int64)
            cnt[n_old + S] = ef
            off = np.zeros(N + 1, np.int64)
            off[1:] = np.cumsum(cnt)
            cand = np.full(int(off[-1]), -1, np.int32)
            for a, u in enumerate(S):
                cand[off[n_old + u]:off[n_old + u + 1]] = W[a]
            pn, pd = prune(D_all, off, cand, Ri, alpha_deg, metric)
            new_nbr = pn[n_old + S]
            new_deg = pd[n_old + S]
            # reverse step for the old nodes that gained in-edges
            row_of = (lambda v: v) if i == 0 else (lambda v: int(rows[v]))
            inc = {}
            for a, u in enumerate(S):
                for v in new_nbr[a, :new_deg[a]]:
                    inc.setdefault(int(v), []).append(n_old + int(u))
            if inc:
                cnt = np.zeros(N, np.int64)
                lists = {}
                for v, us in inc.items():
                    r = row_of(v)
                    lst = list(lay.nbr[r, :lay.deg[r]]) + us
                    lists[v] = lst
                    cnt[v] = len(lst)
                off = np.zeros(N + 1, np.int64)
                off[1:] = np.cumsum(cnt)
                cand = np.empty(int(off[-1]), np.int32)
                for v, lst in lists.items():
                    cand[off[v]:off[v + 1]] = lst
                pn, pd = prune(D_all, off, cand, Ri, alpha_deg, metric)
                for v in lists:
                    r = row_of(v)
                    nbr[r] = pn[v]
                    deg[r] = pd[v]
            gid = np.concatenate([gid, (n_old + S).astype(np.int32)])
            nbr = np.concatenate([nbr, new_nbr])
            deg = np.concatenate([deg, new_deg])
        out[i] = Layer(gid.astype(np.int32), nbr.astype(np.int32), deg.astype(np.int32), Ri)
    return out


# --------------------------------------------------------------------------
def recall_at_k(found_ids, Q, D, k: int, metric: str = "l2", gt=None):
    """Recall@k = |N*(q) cap N(q)| / k (Section 6, performance indicators).

    Reading for ties: a returned id counts when its FP64 distance is at most
    the exact k-th distance; repeated or negative ids count once / never;
    the count is capped at k.  Returns the mean over queries.
    """
    D = _f32(D)
    Q = _f32(Q)
    if gt is None:
        gt = knn(D, k, metric, Q=Q)
    gt_ids, gt_d = gt
    kth = gt_d[:, k - 1]
    total = 0.0
    for qi in range(Q.shape[0]):
        seen = set()
        hit = 0
        for v in found_ids[qi, :k]:
            v = int(v)
            if v < 0 or v in seen:
                continue
            seen.add(v)
            if dist(Q[qi], D[v], metric) <= kth[qi]:
                hit += 1
        total += min(hit, k) / k
    return total / Q.shape[0]


# ------------------------------------------------------------------- K2P
def _prune_scan(D, u: int, cand_row, R: int, ca: float, a60: bool, metric: str, reuse=None):
    """One row of alpha-pruning in plain Python (the Algorithm 3 scan with
    the Section 4.1 rule), optionally with the K2P reuse of Section 5.4:
    ``reuse`` = (C_prev(u), N_prev(u)) as sets.  Returns (kept ids, number
    of occlusion checks that needed s(v, w))."""
    items = sorted({(dist(D[u], D[int(v)], metric), int(v)) for v in cand_row
                    if int(v) >= 0 and int(v) != u})
    out, out_s, checks = [], [], 0
    for suv, v in items:
        if len(out) >= R:
            break
        # K2P: v was a candidate and was kept last time, so no member kept
        # then occluded it; only members new to the kept list are checked
        skip_old = reuse is not None and v in reuse[0] and v in reuse[1]
        occluded = False
        for w, suw in zip(out, out_s):
            if not suw < suv:
                continue
            if skip_old and w in reuse[1]:
                continue
            checks += 1
            svw = dist(D[v], D[w], metric)
            if not svw < suv:
                continue
            if a60 or (suw + svw) - suv < (2.0 * ca) * math.sqrt(suw * svw):
                occluded = True
                break
        if not occluded:
            out.append(v)
            out_s.append(suv)
    return out, checks


def prune_k2p(D, cand_prev, kept_prev, cand, R: int, alpha_deg: float, metric: str = "l2"):
    """K2P of Section 5.4: alpha-pruning of the k-CNA lists ``cand`` (rows of
    C_i(u), -1 padded) that reuses the previous iteration's pruning of the
    same points: for a candidate b that was in C_{i-1}(u) and was kept in
    N_{i-1}(u) (``kept_prev``, the result of pruning C_{i-1}(u) with the same
    rule), the members of N_{i-1}(u) are not checked again.  The pairwise
    occlusion test depends only on u, b and the member, and the list order
    only on s(u, .), so the kept lists are those of plain pruning.  Returns
    (nbr [n][R], deg [n], checks with reuse, checks of the plain scan)."""
    D = _f32(D)
    n = D.shape[0]
    ca, a60 = cos_alpha(alpha_deg), alpha_deg == 60.0
    nbr = np.full((n, R), -1, np.int32)
    deg = np.zeros(n, np.int32)
    reused = plain = 0
    for u in range(n):
        prev = ({int(v) for v in cand_prev[u] if v >= 0}, {int(v) for v in kept_prev[u] if v >= 0})
        out, c = _prune_scan(D, u, cand[u], R, ca, a60, metric, reuse=prev)
        _, c0 = _prune_scan(D, u, cand[u], R, ca, a60, metric)
        nbr[u, :len(out)] = out
        deg[u] = len(out)
        reused += c
        plain += c0
    return nbr, deg, reused, plain


# ---------------------------------------------------- quality examination
def quality_sample_size(n: int, eps: float, l: float = 1.0) -> int:
    """Smallest n_s meeting the bound of Theorem 3 (Section 5.2, quality
    examination): n_s >= (8 + 2 eps) l log n / eps^2, log the natural
    logarithm (the Chernoff bound of the proof is an exponential), so that
    the sample mean of r(u) is within eps / 2 of r(G) / n with probability at
    least 1 - n^-l."""
    if n < 2 or not eps > 0 or not l > 0:
        raise ValueError("need n >= 2, eps > 0, l > 0")
    return int(math.ceil((8.0 + 2.0 * eps) * l * math.log(n) / (eps * eps)))


def kcna_recall(D, cand, k: int, metric: str = "l2", rows=None) -> np.ndarray:
    """r(u) of Section 5.2 for the points ``rows`` (all by default): the
    recall of the first k entries of the k-CNA list C(u) (row u of ``cand``,
    ordered by (s, id), -1 for empty) against the exact k nearest
    neighbours of u other than u.  Reading for ties, as in recall_at_k: an
    entry counts when its FP64 distance to u is at most the exact k-th
    distance; repeated or negative ids count once / never."""
    D = _f32(D)
    cand = np.asarray(cand)
    rows = np.arange(D.shape[0]) if rows is None else np.asarray(rows, np.int64)
    _, gt_d = knn(D, k, metric, rows=rows)
    out = np.empty(rows.shape[0], np.float64)
    for i, u in enumerate(rows):
        kth = gt_d[i, k - 1]
        seen, hit = set(), 0
        for v in cand[u, :k]:
            v = int(v)
            if v < 0 or v == int(u) or v in seen:
                continue
            seen.add(v)
            if dist(D[u], D[v], metric) <= kth:
                hit += 1
        out[i] = min(hit, k) / k
    return out


def estimate_quality(D, cand, k: int, n_s: int, seed: int, metric: str = "l2") -> float:
    """The estimator of Section 5.2: the mean of r(u) over n_s points drawn
    uniformly without replacement (numpy default_rng(seed))."""
    n = np.asarray(D).shape[0]
    sample = np.random.default_rng(seed).choice(n, size=min(n_s, n), replace=False)
    return float(kcna_recall(D, cand, k, metric, rows=np.sort(sample)).mean())


# --------------------------------------------------------------- FP8 rows
# The number format of the FP8-screened queries (a precision form added on
# top of the paper's search, which does not discuss number formats): OCP
# 8-bit floating point E4M3 -- 1 sign bit, 4 exponent bits with bias 7,
# 3 mantissa bits, subnormals, no infinities, S.1111.111 = NaN, largest
# finite value 448.
def fp8_e4m3_decode(codes) -> np.ndarray:
    """Values (float64) of E4M3 codes, from the bit fields; NaN codes give nan."""
    c = np.asarray(codes, np.uint8)
    out = np.empty(c.shape, np.float64)
    for i, b in np.ndenumerate(c):
        b = int(b)
        sign = -1.0 if b & 0x80 else 1.0
        e, m = (b >> 3) & 0xF, b & 0x7
        if e == 0xF and m == 0x7:
            out[i] = math.nan
        elif e == 0:
            out[i] = sign * m * 2.0 ** -9
        else:
            out[i] = sign * (1.0 + m / 8.0) * 2.0 ** (e - 7)
    return out


def _round_half_even(x: float) -> int:
    f = math.floor(x)
    r = x - f
    if r > 0.5 or (r == 0.5 and f % 2 == 1):
        return int(f) + 1
    return int(f)


def fp8_e4m3_encode(values) -> np.ndarray:
    """E4M3 codes of float32 values: nearest representable value, ties to the
    even mantissa, magnitudes of 448 and above saturated to 448; the sign of
    a value that rounds to zero is kept."""
    v = np.asarray(values, np.float32)
    out = np.empty(v.shape, np.uint8)
    for i, x in np.ndenumerate(v):
        x = float(x)
        sign = 0x80 if math.copysign(1.0, x) < 0 else 0
        a = abs(x)
        if a >= 448.0:
            code = 0x7E
        elif a < 2.0 ** -6:
            # subnormals are the multiples of 2^-9; 8 * 2^-9 is the smallest
            # normal, whose code is 0b0001000 = 8 as well
            code = _round_half_even(a * 2.0 ** 9)
        else:
            e = math.frexp(a)[1] - 1  # 2^e <= a < 2^(e + 1)
            q = _round_half_even(a / 2.0 ** (e - 3))  # 8 <= q <= 16
            if q == 16:
                e, q = e + 1, 8
            code = ((e + 7) << 3) | (q - 8)
        out[i] = sign | code
    return out


def fp8_rows(D):
    """FP8 rows of the screened queries: per row scale = max|x| / 448 in
    float32 (1 for a zero row) and the codes of x * float32(1 / scale) (both
    steps in float32)."""
    D = np.asarray(D, np.float32)
    n, d = D.shape
    codes = np.empty((n, d), np.uint8)
    scale = np.empty(n, np.float32)
    for r in range(n):
        mx = np.float32(np.max(np.abs(D[r]))) if d else np.float32(0)
        sc = np.float32(mx / np.float32(448.0)) if mx > 0 else np.float32(1.0)
        inv = np.float32(np.float32(1.0) / sc)
        codes[r] = fp8_e4m3_encode((D[r] * inv).astype(np.float32))
        scale[r] = sc
    return codes, scale

"""Seeded synthetic inputs shaped like the paper's benchmark workloads.

This module is the only code shared by the oracle and the CUDA path.  It
draws points and queries and nothing else: no distance, no ordering, no
pruning or search arithmetic lives here.

The paper evaluates on public image / audio / text embedding sets (Sift1M,
Gist1M, Deep1M, Msong, Crawl, Glove; Section 6, Table 2).  None of them is
used or reproduced; these generators stand in for them with the same n, d
and distance family:

* ``mixture_int``   -- Gaussian mixture of isotropic clusters with centres
  drawn U[0,255]^d, values rounded to integers and clipped to [0,255]
  (Sift-like byte-valued descriptors), stored as float32.
* ``mixture_float`` -- Gaussian mixture with centres U[0,1]^d, no rounding
  (Gist-like real descriptors).
* ``unit_gaussian`` -- i.i.d. N(0, I) rows normalised to unit length
  (Deep/Glove-like embeddings under cosine distance).
* ``sphere_mixture`` -- clusters on the unit sphere: normalise(c + s*N(0,I))
  with c a normalised N(0, I) draw.

Every generator is deterministic in its seed (numpy ``default_rng``); rows
are produced in chunks so that 1M x 960 inputs do not need a float64 copy
of the whole matrix.
"""
from __future__ import annotations

import numpy as np

_CHUNK = 1 << 16


def _labels(rng: np.random.Generator, n: int, n_clusters: int) -> np.ndarray:
    return rng.integers(0, n_clusters, size=n)


def mixture_int(n: int, d: int, n_clusters: int, seed: int, sigma: float = 20.0,
                centres: np.ndarray | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Byte-valued Gaussian mixture; returns (points float32[n][d], centres)."""
    rng = np.random.default_rng(seed)
    if centres is None:
        centres = rng.uniform(0.0, 255.0, size=(n_clusters, d))
    lab = _labels(rng, n, centres.shape[0])
    out = np.empty((n, d), dtype=np.float32)
    for a in range(0, n, _CHUNK):
        b = min(n, a + _CHUNK)
        x = centres[lab[a:b]] + rng.normal(0.0, sigma, size=(b - a, d))
        out[a:b] = np.clip(np.rint(x), 0.0, 255.0)
    return out, centres


def mixture_float(n: int, d: int, n_clusters: int, seed: int, sigma: float = 0.1,
                  centres: np.ndarray | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Real-valued Gaussian mixture around U[0,1]^d centres (no clipping)."""
    rng = np.random.default_rng(seed)
    if centres is None:
        centres = rng.uniform(0.0, 1.0, size=(n_clusters, d))
    lab = _labels(rng, n, centres.shape[0])
    out = np.empty((n, d), dtype=np.float32)
    for a in range(0, n, _CHUNK):
        b = min(n, a + _CHUNK)
        out[a:b] = centres[lab[a:b]] + rng.normal(0.0, sigma, size=(b - a, d))
    return out, centres


def _normalise_rows(x: np.ndarray) -> np.ndarray:
    nrm = np.sqrt(np.sum(x * x, axis=1, keepdims=True))
    nrm[nrm == 0.0] = 1.0
    return x / nrm


def unit_gaussian(n: int, d: int, seed: int) -> np.ndarray:
    """Rows of N(0, I) scaled to unit L2 norm, float32."""
    rng = np.random.default_rng(seed)
    out = np.empty((n, d), dtype=np.float32)
    for a in range(0, n, _CHUNK):
        b = min(n, a + _CHUNK)
        out[a:b] = _normalise_rows(rng.normal(0.0, 1.0, size=(b - a, d)))
    return out


def sphere_mixture(n: int, d: int, n_clusters: int, seed: int, sigma: float | None = None,
                   centres: np.ndarray | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Clusters on the unit sphere; sigma defaults to 0.5/sqrt(d)."""
    rng = np.random.default_rng(seed)
    if sigma is None:
        sigma = 0.5 / np.sqrt(d)
    if centres is None:
        centres = _normalise_rows(rng.normal(0.0, 1.0, size=(n_clusters, d)))
    lab = _labels(rng, n, centres.shape[0])
    out = np.empty((n, d), dtype=np.float32)
    for a in range(0, n, _CHUNK):
        b = min(n, a + _CHUNK)
        x = centres[lab[a:b]] + rng.normal(0.0, sigma, size=(b - a, d))
        out[a:b] = _normalise_rows(x)
    return out, centres


# ---------------------------------------------------------------------------
# The five workloads (points and queries).  Seeds: points 1234 + c, queries
# 5678 + c for workload number c.  Queries reuse the points' cluster centres.
# ---------------------------------------------------------------------------

WORKLOADS = {
    1: dict(name="rng-fp32-10k-d128", n=10_000, d=128, clusters=32, kind="int",
            metric="l2", K=20, L=100, R=32, nq=100, k=10, beams=[64]),
    2: dict(name="rng-1m-d128", n=1_000_000, d=128, clusters=1024, kind="int",
            metric="l2", K=64, L=200, R=32, nq=10_000, k=10,
            beams=[32, 48, 64, 96, 128, 192, 256]),
    3: dict(name="rng-bf16-1m-d960", n=1_000_000, d=960, clusters=512, kind="float",
            metric="l2", K=64, L=200, R=32, nq=1_000, k=10, beams=[64, 128, 256]),
    4: dict(name="nswg-1m-d96-cosine", n=1_000_000, d=96, clusters=0, kind="unit",
            metric="cosine", K=64, L=200, R=32, M=16, nq=10_000, k=10,
            beams=[32, 64, 128, 256]),
    5: dict(name="serve-2m-d384-ip", n=2_000_000, d=384, clusters=4096, kind="sphere",
            metric="ip", K=64, L=200, R=32, M=16, nq=10_000, k=10, beams=[64, 128, 256]),
}


def make(kind: str, n: int, d: int, clusters: int, seed: int, nq: int, qseed: int):
    """Points and queries for one workload kind; returns (D, Q)."""
    if kind == "int":
        D, c = mixture_int(n, d, clusters, seed)
        Q, _ = mixture_int(nq, d, clusters, qseed, centres=c)
    elif kind == "float":
        D, c = mixture_float(n, d, clusters, seed)
        Q, _ = mixture_float(nq, d, clusters, qseed, centres=c)
    elif kind == "unit":
        D = unit_gaussian(n, d, seed)
        Q = unit_gaussian(nq, d, qseed)
    elif kind == "sphere":
        D, c = sphere_mixture(n, d, clusters, seed)
        Q, _ = sphere_mixture(nq, d, clusters, qseed, centres=c)
    else:
        raise ValueError(kind)
    return D, Q


def inserts(c: int, m: int) -> np.ndarray:
    """m further points of workload ``c`` for insertion (same cluster centres
    as its points, seed 9012 + c)."""
    w = WORKLOADS[c]
    kind, d, k, seed = w["kind"], w["d"], w["clusters"], 9012 + c
    if kind == "int":
        return mixture_int(m, d, k, seed, centres=mixture_int(1, d, k, 1234 + c)[1])[0]
    if kind == "float":
        return mixture_float(m, d, k, seed, centres=mixture_float(1, d, k, 1234 + c)[1])[0]
    if kind == "unit":
        return unit_gaussian(m, d, seed)
    return sphere_mixture(m, d, k, seed, centres=sphere_mixture(1, d, k, 1234 + c)[1])[0]


def workload(c: int, n: int | None = None, nq: int | None = None):
    """(D, Q, params) of workload ``c``; ``n``/``nq`` shrink it for tests."""
    w = dict(WORKLOADS[c])
    if n is not None:
        w["n"] = n
    if nq is not None:
        w["nq"] = nq
    D, Q = make(w["kind"], w["n"], w["d"], w["clusters"], 1234 + c, w["nq"], 5678 + c)
    return D, Q, w

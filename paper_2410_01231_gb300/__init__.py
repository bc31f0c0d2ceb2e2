"""Python binding of libpg: proximity-graph construction and search on one
GB300 GPU, after the framework of arXiv 2410.01231.

Argument marshalling only: every step runs in the CUDA kernels of libpg.so
(built in-tree from ``csrc/`` for sm_103a).  Importing this package loads the
library and raises if it is missing -- there is no CPU fallback.  Torch
tensors provide device memory and the stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import _build

_LIB_PATH = _build.LIB

if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libpg.so is not built ({_LIB_PATH}); run paper_2410_01231_gb300._build.build()"
                      " or __graft_entry__.build()")

_lib = C.CDLL(_LIB_PATH)

METRIC = {"l2": 0, "cosine": 1, "ip": 2}
# pool width of the descent through the upper layers of a hierarchical index
# (1 is the paper's greedy routing; 16 enters the query's cluster far more
# reliably on well-separated data)
UPPER_BEAM = 16
PRECISION = {"fp32": 0, "bf16": 1, "fp8": 2}
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "TIMEOUT", 5: "CAPACITY", 6: "BUDGET",
          7: "INTERNAL", 8: "DEVICE_CHECK", 9: "IO"}

P = C.c_void_p
i32, i64, dbl, u64 = C.c_int32, C.c_int64, C.c_double, C.c_uint64


class BuildParams(C.Structure):
    _fields_ = [("metric", C.c_int), ("precision", C.c_int), ("K", i32), ("L", i32), ("R", i32),
                ("M", i32), ("alpha_deg", dbl), ("alpha_final_deg", dbl), ("iters", i32),
                ("connect_final", i32), ("route_layers", i32), ("seed", u64),
                ("reuse_pruning", i32), ("quality_target", dbl), ("quality_eps", dbl),
                ("quality_k", i32), ("connect_replace", i32), ("knn_descent_iters", i32)]


class PruneStats(C.Structure):
    _fields_ = [(name, i64) for name in ("rows", "candidates", "scanned", "occlusion_tests",
                                         "fp64_rechecks", "fp64_flips", "edges", "long_rows",
                                         "near_ties")]


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("pg_default_params", None, [P])
_sig("pg_ctx_create", C.c_int, [P, C.c_size_t, P])
_sig("pg_ctx_destroy", None, [P])
_sig("pg_last_error", C.c_char_p, [P])
_sig("pg_ctx_sync", C.c_int, [P])
_sig("pg_ctx_launches", i64, [P])
_sig("pg_build_knn", C.c_int, [P, P, i64, i32, C.c_int, i32, C.c_int, P, P])
_sig("pg_knn_query", C.c_int, [P, P, i64, i32, C.c_int, P, i64, i32, C.c_int, P, P])
_sig("pg_prune", C.c_int, [P, P, i64, i32, C.c_int, P, P, i32, dbl, C.c_int, P, P, P])
_sig("pg_kcna_recall", C.c_int, [P, P, i64, i32, C.c_int, P, i32, i32, P, i64, P, P])
_sig("pg_quality_sample_size", i64, [i64, dbl, dbl])
_sig("pg_quality_sample", C.c_int, [i64, i64, u64, P])
_sig("pg_index_quality", C.c_int, [P, P, P, P])
_sig("pg_connect_replace", C.c_int, [P, P, i64, i32, C.c_int, P, P, i32, i64, P, P])
_sig("pg_knn_descent", C.c_int, [P, P, i64, i32, C.c_int, i32, i32, P, u64, P, P, P])
_sig("pg_prune_k2p", C.c_int, [P, P, i64, i32, C.c_int, P, P, P, P, i32, i32, dbl, C.c_int, P, P,
                               P])
_sig("pg_reverse_union", C.c_int, [P, P, P, i64, i32, P, P, i64, P])
_sig("pg_medoid", C.c_int, [P, P, i64, i32, C.c_int, P])
_sig("pg_connect", C.c_int, [P, P, i64, i32, C.c_int, P, P, i32, i64, P])
_sig("pg_acquire_candidates", C.c_int, [P, P, i64, i32, C.c_int, P, P, i32, i32, C.c_int, P])
_sig("pg_search_graph", C.c_int, [P, P, i64, i32, C.c_int, P, P, i32, P, P, i64, P, i32, i32,
                                  C.c_int, P, P])
_sig("pg_build_rng", C.c_int, [P, P, i64, i32, P, P])
_sig("pg_build_nswg", C.c_int, [P, P, i64, i32, P, P])
_sig("pg_build_rng_host", C.c_int, [P, P, i64, i32, P, P, P, P])
_sig("pg_measure_fp32_peak", C.c_int, [P, P])
_sig("pg_search", C.c_int, [P, P, P, i64, i32, i32, i32, i32, C.c_int, P, P])
_sig("pg_search_host", C.c_int, [P, P, P, i64, i32, i32, i32, i32, C.c_int, P, P])
_sig("pg_index_destroy", None, [P])
_sig("pg_index_info", C.c_int, [P, P, P, P, P])
_sig("pg_index_layer", C.c_int, [P, i32, P, P, P, P, P])
_sig("pg_index_phase_seconds", C.c_int, [P, P])
_sig("pg_index_export_layer", C.c_int, [P, P, i32, P, P, P])
_sig("pg_ctx_set_timing", C.c_int, [P, C.c_int])
_sig("pg_ctx_set_tie_count", C.c_int, [P, C.c_int])
_sig("pg_ctx_set_autotune", C.c_int, [P, C.c_int])
_sig("pg_autotune_report", i64, [P, i64])
_sig("pg_ctx_kernel_time", C.c_int, [P, C.c_char_p, P, P])
_sig("pg_ctx_counter", C.c_int, [P, C.c_char_p, P])
_sig("pg_ctx_kernel_work", C.c_int, [P, C.c_char_p, P])
_sig("pg_prune_noalloc", C.c_int, [P, P, i64, i32, C.c_int, P, P, i32, dbl, P, P])
_sig("pg_index_reserve", C.c_int, [P, P, i64])
_sig("pg_index_insert", C.c_int, [P, P, P, i64, i32, i32])
_sig("pg_serve_start", C.c_int, [P, P, i32, i32, P])
_sig("pg_serve_submit_query", C.c_int, [P, P, i64, i32, i32, i32, P, P, P])
_sig("pg_serve_submit_insert", C.c_int, [P, P, i64, i32, i32, P])
_sig("pg_serve_wait", C.c_int, [P, i64, dbl, P])
_sig("pg_serve_stats", C.c_int, [P, P, i32])
_sig("pg_serve_stop", C.c_int, [P])
_sig("pg_serve_set_queue_limit", C.c_int, [P, i64])
_sig("pg_serve_set_budget", C.c_int, [P, i64])
_sig("pg_serve_latency", C.c_int, [P, i64, P])
_sig("pg_serve_set_precision", C.c_int, [P, C.c_int])
_sig("pg_encode_fp8", C.c_int, [P, P, i64, i32, P, P])
_sig("pg_levels", C.c_int, [i64, u64, i32, P])
_sig("pg_selftest_wait_timeout", C.c_int, [P, dbl])
_sig("pg_index_params", C.c_int, [P, P, P])
_sig("pg_index_save", C.c_int, [P, P, C.c_char_p])
_sig("pg_index_load", C.c_int, [P, C.c_char_p, P])
_sig("pg_index_file_check", C.c_int, [C.c_char_p, P, P, P, C.c_char_p, C.c_size_t])
_sig("pg_serve_simulate", C.c_int, [i32, i32, i64, i32, P, P, P, i32, i64, P, P, P, P, P, P])

EXPORTS = ["pg_default_params", "pg_ctx_create", "pg_ctx_destroy", "pg_last_error", "pg_ctx_sync",
           "pg_ctx_launches", "pg_build_knn", "pg_knn_query", "pg_prune", "pg_reverse_union",
           "pg_medoid", "pg_connect", "pg_acquire_candidates", "pg_search_graph", "pg_build_rng",
           "pg_build_rng_host", "pg_measure_fp32_peak", "pg_prune_k2p",
           "pg_kcna_recall", "pg_connect_replace", "pg_knn_descent", "pg_quality_sample_size", "pg_quality_sample", "pg_index_quality",
           "pg_build_nswg", "pg_search", "pg_search_host", "pg_index_destroy", "pg_index_info",
           "pg_index_layer", "pg_index_phase_seconds", "pg_index_export_layer",
           "pg_ctx_set_timing", "pg_ctx_set_tie_count", "pg_ctx_set_autotune",
           "pg_autotune_report", "pg_ctx_kernel_time", "pg_ctx_counter",
           "pg_ctx_kernel_work", "pg_prune_noalloc", "pg_index_reserve", "pg_index_insert",
           "pg_serve_start", "pg_serve_submit_query", "pg_serve_submit_insert", "pg_serve_wait",
           "pg_serve_stats", "pg_serve_stop", "pg_serve_set_queue_limit",
           "pg_selftest_wait_timeout", "pg_index_params", "pg_index_save", "pg_index_load",
           "pg_index_file_check", "pg_serve_simulate",
           "pg_serve_set_budget", "pg_serve_latency", "pg_serve_set_precision",
           "pg_encode_fp8", "pg_levels"]


class PGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"pg status {STATUS.get(status, status)}: {msg}")
        self.status = status


def _ptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def _dev(t: torch.Tensor, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return t.contiguous()


class Context:
    """A libpg context bound to the current device and a CUDA stream."""

    def __init__(self, stream: torch.cuda.Stream | None = None, hbm_budget_bytes: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("libpg needs a CUDA device")
        self.stream = stream or torch.cuda.current_stream()
        self.device = torch.device("cuda", torch.cuda.current_device())
        h = C.c_void_p()
        st = _lib.pg_ctx_create(C.c_void_p(self.stream.cuda_stream), hbm_budget_bytes, C.byref(h))
        if st != 0:
            raise PGError(st, "pg_ctx_create")
        self._h = h

    def _check(self, st, what):
        if st != 0:
            raise PGError(st, f"{what}: {_lib.pg_last_error(self._h).decode()}")

    def sync(self):
        self._check(_lib.pg_ctx_sync(self._h), "sync")

    @property
    def launches(self) -> int:
        return int(_lib.pg_ctx_launches(self._h))

    def set_timing(self, enable: bool = True):
        """Enable CUDA-event timing of the main kernels (resets totals)."""
        self._check(_lib.pg_ctx_set_timing(self._h, 1 if enable else 0), "pg_ctx_set_timing")

    def set_tie_count(self, enable: bool = True):
        """Count pruning decisions with relative margin below 1e-5 (pg_ctx_set_tie_count)."""
        self._check(_lib.pg_ctx_set_tie_count(self._h, 1 if enable else 0),
                    "pg_ctx_set_tie_count")

    def set_autotune(self, enable: bool = True):
        """Launch configurations of the prune / search kernels chosen by timing
        (pg_ctx_set_autotune)."""
        self._check(_lib.pg_ctx_set_autotune(self._h, 1 if enable else 0), "pg_ctx_set_autotune")

    def kernel_time(self, name: str):
        """(total device ms, launches) of a timed kernel since the last reset."""
        ms, cnt = C.c_double(), C.c_int64()
        self._check(_lib.pg_ctx_kernel_time(self._h, name.encode(), C.byref(ms), C.byref(cnt)),
                    "pg_ctx_kernel_time")
        return ms.value, cnt.value

    def kernel_work(self, name: str) -> float:
        """Algorithmic work (flops) of the timed launches of `name`."""
        v = C.c_double()
        self._check(_lib.pg_ctx_kernel_work(self._h, name.encode(), C.byref(v)),
                    "pg_ctx_kernel_work")
        return v.value

    def measure_fp32_peak(self) -> float:
        """Measured FP32 FMA throughput of the device in TFLOP/s (pg_measure_fp32_peak)."""
        v = C.c_double()
        self._check(_lib.pg_measure_fp32_peak(self._h, C.byref(v)), "pg_measure_fp32_peak")
        return v.value

    def selftest_wait_timeout(self, seconds: float = 0.2):
        """Bounded-wait failure path (pg_selftest_wait_timeout): raises PGError TIMEOUT."""
        self._check(_lib.pg_selftest_wait_timeout(self._h, float(seconds)),
                    "pg_selftest_wait_timeout")

    def counter(self, name: str) -> int:
        """Cumulative counter (pg_ctx_counter): "connect_edges", "connect_full_rounds",
        "connect_conflicts", "search_expansions", "search_evaluations", "prune_rows",
        "prune_candidates", "prune_scanned", "prune_occlusion_tests", "prune_edges",
        "prune_fp64_rechecks", "prune_fp64_flips", "prune_near_ties", "search_bytes",
        "prune_bytes"."""
        v = C.c_int64()
        self._check(_lib.pg_ctx_counter(self._h, name.encode(), C.byref(v)), "pg_ctx_counter")
        return v.value

    def close(self):
        if getattr(self, "_h", None):
            _lib.pg_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h


def autotune_report() -> str:
    """The autotuner's table (pg_autotune_report)."""
    need = int(_lib.pg_autotune_report(None, 0))
    buf = C.create_string_buffer(max(need, 1))
    _lib.pg_autotune_report(buf, need)
    return buf.value.decode()


def default_params(**kw) -> BuildParams:
    p = BuildParams()
    _lib.pg_default_params(C.byref(p))
    names = {f for f, _ in BuildParams._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"unknown build parameter {k!r}")
        if k == "metric":
            v = METRIC[v] if isinstance(v, str) else v
        if k == "precision":
            v = PRECISION[v] if isinstance(v, str) else v
        setattr(p, k, v)
    return p


# --------------------------------------------------------------- steps
def index_file_check(path: str) -> dict:
    """Host-only check of an index file (pg_index_file_check, no GPU needed):
    {"n", "d", "n_layers"} of a valid file, else PGError with the reason."""
    n, d, nl = C.c_int64(), C.c_int32(), C.c_int32()
    msg = C.create_string_buffer(256)
    st = _lib.pg_index_file_check(os.fsencode(path), C.byref(n), C.byref(d), C.byref(nl), msg,
                                  len(msg))
    if st != 0:
        raise PGError(st, f"pg_index_file_check: {msg.value.decode()}")
    return dict(n=n.value, d=d.value, n_layers=nl.value)


def levels(n: int, seed: int, M: int) -> np.ndarray:
    """Layer of every point id as the NSWG build draws it (pg_levels, host only)."""
    out = np.empty(n, np.int32)
    st = _lib.pg_levels(n, seed, M, out.ctypes.data_as(C.c_void_p))
    if st != 0:
        raise PGError(st, "pg_levels")
    return out


def encode_fp8(ctx: Context, D: torch.Tensor):
    """FP8 E4M3 rows of D as the screened search uses them (pg_encode_fp8):
    (codes uint8 [n][d], scale float32 [n])."""
    D = _dev(D, torch.float32, "D")
    n, d = D.shape
    codes = torch.empty((n, d), dtype=torch.uint8, device=D.device)
    scale = torch.empty(n, dtype=torch.float32, device=D.device)
    ctx._check(_lib.pg_encode_fp8(ctx.handle, _ptr(D), n, d, _ptr(codes), _ptr(scale)),
               "pg_encode_fp8")
    return codes, scale


def build_knn(ctx: Context, D: torch.Tensor, K: int, metric="l2", precision="fp32"):
    """Exact K-NN graph: (ids int32 [n][K], dist float32 [n][K])."""
    D = _dev(D, torch.float32, "D")
    n, d = D.shape
    ids = torch.empty((n, K), dtype=torch.int32, device=D.device)
    dist = torch.empty((n, K), dtype=torch.float32, device=D.device)
    ctx._check(_lib.pg_build_knn(ctx.handle, _ptr(D), n, d, METRIC[metric], K,
                                 PRECISION[precision], _ptr(ids), _ptr(dist)), "pg_build_knn")
    return ids, dist


def knn_descent(ctx: Context, D: torch.Tensor, K: int, iters: int, init=None, seed: int = 0,
                metric="l2"):
    """pg_knn_descent: approximate KNNG by 2-hop refinement; returns
    (ids [n][K], dist [n][K], entries entering the lists per iteration)."""
    D = _dev(D, torch.float32, "D")
    n, d = D.shape
    if init is not None:
        init = _dev(init, torch.int32, "init")
    ids = torch.empty((n, K), dtype=torch.int32, device=D.device)
    dist = torch.empty((n, K), dtype=torch.float32, device=D.device)
    upd = (C.c_int64 * max(iters, 1))()
    ctx._check(_lib.pg_knn_descent(ctx.handle, _ptr(D), n, d, METRIC[metric], K, iters,
                                   _ptr(init), int(seed), _ptr(ids), _ptr(dist), upd),
               "pg_knn_descent")
    return ids, dist, [int(upd[i]) for i in range(iters)]


def knn_query(ctx: Context, D: torch.Tensor, Q: torch.Tensor, k: int, metric="l2",
              precision="fp32"):
    D = _dev(D, torch.float32, "D")
    Q = _dev(Q, torch.float32, "Q")
    ids = torch.empty((Q.shape[0], k), dtype=torch.int32, device=D.device)
    dist = torch.empty((Q.shape[0], k), dtype=torch.float32, device=D.device)
    ctx._check(_lib.pg_knn_query(ctx.handle, _ptr(D), D.shape[0], D.shape[1], METRIC[metric],
                                 _ptr(Q), Q.shape[0], k, PRECISION[precision], _ptr(ids),
                                 _ptr(dist)), "pg_knn_query")
    return ids, dist


def prune(ctx: Context, D, off, cand, R: int, alpha_deg: float, metric="l2", precision="fp32",
          stats: bool = False):
    """alpha-pruning of CSR candidate rows: (nbr [n][R], deg [n][, stats])."""
    D = _dev(D, torch.float32, "D")
    off = _dev(off, torch.int64, "off")
    cand = _dev(cand, torch.int32, "cand")
    n, d = D.shape
    nbr = torch.empty((n, R), dtype=torch.int32, device=D.device)
    deg = torch.empty(n, dtype=torch.int32, device=D.device)
    ps = PruneStats()
    ctx._check(_lib.pg_prune(ctx.handle, _ptr(D), n, d, METRIC[metric], _ptr(off), _ptr(cand), R,
                             float(alpha_deg), PRECISION[precision], _ptr(nbr), _ptr(deg),
                             C.byref(ps) if stats else None), "pg_prune")
    if stats:
        return nbr, deg, {k: int(getattr(ps, k)) for k, _ in PruneStats._fields_}
    return nbr, deg


def kcna_recall(ctx: Context, D, cand, k: int, sample, metric="l2"):
    """pg_kcna_recall: (r(u) for each sampled u as a float64 device tensor,
    their mean) for the k-CNA rows cand [n][L] (Section 5.2)."""
    D = _dev(D, torch.float32, "D")
    cand = _dev(cand, torch.int32, "cand")
    sample = _dev(sample, torch.int32, "sample")
    n, d = D.shape
    ns = sample.shape[0]
    rec = torch.empty(ns, dtype=torch.float64, device=D.device)
    mean = C.c_double()
    ctx._check(_lib.pg_kcna_recall(ctx.handle, _ptr(D), n, d, METRIC[metric], _ptr(cand),
                                   cand.shape[1], k, _ptr(sample), ns, _ptr(rec), C.byref(mean)),
               "pg_kcna_recall")
    return rec, mean.value


def quality_sample_size(n: int, eps: float, l: float = 1.0) -> int:
    """Theorem 3's sample size (pg_quality_sample_size, host only)."""
    return int(_lib.pg_quality_sample_size(int(n), float(eps), float(l)))


def quality_sample(n: int, ns: int, seed: int) -> np.ndarray:
    """The builds' sample of ns distinct ids of [0, n) (pg_quality_sample, host only)."""
    out = np.empty(max(ns, 1), np.int32)
    st = _lib.pg_quality_sample(int(n), int(ns), int(seed), out.ctypes.data)
    if st != 0:
        raise PGError(st, "pg_quality_sample")
    return out[:ns]


def prune_k2p(ctx: Context, D, off, cand, prev_nbr, prev_deg, R: int, alpha_deg: float,
              metric="l2", precision="fp32", stats: bool = False):
    """pg_prune_k2p: alpha-pruning that reuses an earlier pruning of the same
    points (prev_nbr [n][prev_R], prev_deg [n]) as Section 5.4's K2P."""
    D = _dev(D, torch.float32, "D")
    off = _dev(off, torch.int64, "off")
    cand = _dev(cand, torch.int32, "cand")
    prev_nbr = _dev(prev_nbr, torch.int32, "prev_nbr")
    prev_deg = _dev(prev_deg, torch.int32, "prev_deg")
    n, d = D.shape
    nbr = torch.empty((n, R), dtype=torch.int32, device=D.device)
    deg = torch.empty(n, dtype=torch.int32, device=D.device)
    ps = PruneStats()
    ctx._check(_lib.pg_prune_k2p(ctx.handle, _ptr(D), n, d, METRIC[metric], _ptr(off), _ptr(cand),
                                 _ptr(prev_nbr), _ptr(prev_deg), prev_nbr.shape[1], R,
                                 float(alpha_deg), PRECISION[precision], _ptr(nbr), _ptr(deg),
                                 C.byref(ps) if stats else None), "pg_prune_k2p")
    if stats:
        return nbr, deg, {k: int(getattr(ps, k)) for k, _ in PruneStats._fields_}
    return nbr, deg


def prune_noalloc(D, off, cand, R: int, alpha_deg: float, metric="l2", stream=None):
    """pg_prune_noalloc: the pruning step without any device allocation
    inside the library (fixed scratch; n <= 2^20; synchronous)."""
    D = _dev(D, torch.float32, "D")
    off = _dev(off, torch.int64, "off")
    cand = _dev(cand, torch.int32, "cand")
    n, d = D.shape
    nbr = torch.empty((n, R), dtype=torch.int32, device=D.device)
    deg = torch.empty(n, dtype=torch.int32, device=D.device)
    s = (stream or torch.cuda.current_stream()).cuda_stream
    st = _lib.pg_prune_noalloc(C.c_void_p(s), _ptr(D), n, d, METRIC[metric], _ptr(off),
                               _ptr(cand), R, float(alpha_deg), _ptr(nbr), _ptr(deg))
    if st != 0:
        raise PGError(st, "pg_prune_noalloc")
    return nbr, deg


def reverse_union(ctx: Context, nbr, deg):
    nbr = _dev(nbr, torch.int32, "nbr")
    deg = _dev(deg, torch.int32, "deg")
    n, R = nbr.shape
    off = torch.empty(n + 1, dtype=torch.int64, device=nbr.device)
    ids = torch.empty(2 * n * R, dtype=torch.int32, device=nbr.device)
    tot = C.c_int64()
    ctx._check(_lib.pg_reverse_union(ctx.handle, _ptr(nbr), _ptr(deg), n, R, _ptr(off), _ptr(ids),
                                     2 * n * R, C.byref(tot)), "pg_reverse_union")
    return off, ids[: tot.value]


def medoid(ctx: Context, D, metric="l2") -> int:
    D = _dev(D, torch.float32, "D")
    ep = C.c_int64()
    ctx._check(_lib.pg_medoid(ctx.handle, _ptr(D), D.shape[0], D.shape[1], METRIC[metric],
                              C.byref(ep)), "pg_medoid")
    return int(ep.value)


def connect(ctx: Context, D, nbr, deg, ep: int, metric="l2") -> int:
    """In place on nbr/deg; returns the number of edges added."""
    D = _dev(D, torch.float32, "D")
    if not (nbr.is_contiguous() and deg.is_contiguous()):
        raise ValueError("nbr/deg must be contiguous (updated in place)")
    n, R = nbr.shape
    added = C.c_int64()
    ctx._check(_lib.pg_connect(ctx.handle, _ptr(D), n, D.shape[1], METRIC[metric], _ptr(nbr),
                               _ptr(deg), R, ep, C.byref(added)), "pg_connect")
    return int(added.value)


def connect_replace(ctx: Context, D, nbr, deg, ep: int, metric="l2"):
    """pg_connect_replace, in place on nbr/deg: (edges added, replacements)."""
    D = _dev(D, torch.float32, "D")
    if not (nbr.is_contiguous() and deg.is_contiguous()):
        raise ValueError("nbr/deg must be contiguous (updated in place)")
    n, R = nbr.shape
    added, rep = C.c_int64(), C.c_int64()
    ctx._check(_lib.pg_connect_replace(ctx.handle, _ptr(D), n, D.shape[1], METRIC[metric],
                                       _ptr(nbr), _ptr(deg), R, ep, C.byref(added),
                                       C.byref(rep)), "pg_connect_replace")
    return int(added.value), int(rep.value)


def acquire_candidates(ctx: Context, D, nbr, deg, L: int, metric="l2", precision="fp32"):
    D = _dev(D, torch.float32, "D")
    nbr = _dev(nbr, torch.int32, "nbr")
    deg = _dev(deg, torch.int32, "deg")
    n, d = D.shape
    cand = torch.empty((n, L), dtype=torch.int32, device=D.device)
    ctx._check(_lib.pg_acquire_candidates(ctx.handle, _ptr(D), n, d, METRIC[metric], _ptr(nbr),
                                          _ptr(deg), nbr.shape[1], L, PRECISION[precision],
                                          _ptr(cand)), "pg_acquire_candidates")
    return cand


def search_graph(ctx: Context, D, nbr, deg, Q, starts, k: int, L: int, metric="l2", rows=None,
                 precision="fp32"):
    D = _dev(D, torch.float32, "D")
    nbr = _dev(nbr, torch.int32, "nbr")
    deg = _dev(deg, torch.int32, "deg")
    Q = _dev(Q, torch.float32, "Q")
    starts = _dev(starts, torch.int32, "starts")
    rows = None if rows is None else _dev(rows, torch.int32, "rows")
    nq = Q.shape[0]
    ids = torch.empty((nq, k), dtype=torch.int32, device=D.device)
    dist = torch.empty((nq, k), dtype=torch.float32, device=D.device)
    ctx._check(_lib.pg_search_graph(ctx.handle, _ptr(D), D.shape[0], D.shape[1], METRIC[metric],
                                    _ptr(nbr), _ptr(deg), nbr.shape[1], _ptr(rows), _ptr(Q), nq,
                                    _ptr(starts), k, L, PRECISION[precision], _ptr(ids),
                                    _ptr(dist)), "pg_search_graph")
    return ids, dist


# --------------------------------------------------------------- index
class Index:
    """A built graph index (owned by libpg; D must stay alive unless the index
    holds its own copy of the points: after reserve() or load())."""

    def __init__(self, ctx: Context, handle, D: torch.Tensor | None, metric: str,
                 device: torch.device | None = None):
        self.ctx, self._h, self.D, self.metric = ctx, handle, D, metric
        self.device = D.device if D is not None else device

    @classmethod
    def load(cls, ctx: Context, path: str):
        """Read an index file written by save() (pg_index_load): checked in full on
        the host, then copied to the context's device, points included."""
        h = C.c_void_p()
        ctx._check(_lib.pg_index_load(ctx.handle, os.fsencode(path), C.byref(h)),
                   "pg_index_load")
        p, d = BuildParams(), C.c_int32()
        _lib.pg_index_params(h, C.byref(p), C.byref(d))
        metric = {v: k for k, v in METRIC.items()}[p.metric]
        return cls(ctx, h, None, metric, ctx.device)

    def save(self, path: str):
        """Write the index, its build parameters and its points to `path` (pg_index_save)."""
        self.ctx._check(_lib.pg_index_save(self.ctx.handle, self._h, os.fsencode(path)),
                        "pg_index_save")

    def params(self):
        """Build parameters (a BuildParams structure) and dimension of the index."""
        p, d = BuildParams(), C.c_int32()
        st = _lib.pg_index_params(self._h, C.byref(p), C.byref(d))
        if st != 0:
            raise PGError(st, "pg_index_params")
        return p, d.value

    @classmethod
    def build_rng(cls, ctx: Context, D: torch.Tensor, **params):
        return cls._build(ctx, D, "pg_build_rng", params)

    @classmethod
    def build_rng_host(cls, ctx: Context, D: torch.Tensor, nbr: torch.Tensor, deg: torch.Tensor,
                       keep: bool = False, **params):
        """pg_build_rng_host: D [n][d] float32 in HOST memory (pinned or not) is
        uploaded, built and the base graph written to the HOST tensors nbr
        [n][R] and deg [n] (int32).  Returns an Index owning its points when
        keep, else None."""
        if D.is_cuda or nbr.is_cuda or deg.is_cuda:
            raise ValueError("build_rng_host takes host tensors")
        if D.dtype != torch.float32 or not D.is_contiguous() or D.dim() != 2:
            raise ValueError("D must be a contiguous float32 [n][d] host tensor")
        p = default_params(**params)
        n = D.shape[0]
        if (nbr.dtype != torch.int32 or deg.dtype != torch.int32 or tuple(nbr.shape) != (n, p.R)
                or tuple(deg.shape) != (n,) or not nbr.is_contiguous()):
            raise ValueError("nbr must be int32 [n][R] and deg int32 [n], contiguous")
        h = C.c_void_p()
        ctx._check(_lib.pg_build_rng_host(ctx.handle, C.c_void_p(D.data_ptr()), n, D.shape[1],
                                          C.byref(p), C.c_void_p(nbr.data_ptr()),
                                          C.c_void_p(deg.data_ptr()),
                                          C.byref(h) if keep else None), "pg_build_rng_host")
        if not keep:
            return None
        metric = {v: k for k, v in METRIC.items()}[p.metric]
        return cls(ctx, h, None, metric, ctx.device)

    @classmethod
    def build_nswg(cls, ctx: Context, D: torch.Tensor, **params):
        return cls._build(ctx, D, "pg_build_nswg", params)

    @classmethod
    def _build(cls, ctx, D, fn, params):
        D = _dev(D, torch.float32, "D")
        p = default_params(**params)
        h = C.c_void_p()
        ctx._check(getattr(_lib, fn)(ctx.handle, _ptr(D), D.shape[0], D.shape[1], C.byref(p),
                                     C.byref(h)), fn)
        metric = {v: k for k, v in METRIC.items()}[p.metric]
        return cls(ctx, h, D, metric)

    def info(self):
        nl, n, et, eb = C.c_int32(), C.c_int64(), C.c_int64(), C.c_int64()
        _lib.pg_index_info(self._h, C.byref(nl), C.byref(n), C.byref(et), C.byref(eb))
        return dict(n_layers=nl.value, n=n.value, ep_top=et.value, ep_base=eb.value)

    def layer(self, i: int):
        """(gid, nbr, deg) of layer i as new device tensors (gid of layer 0 is 0..n-1)."""
        cnt, R = C.c_int64(), C.c_int32()
        st = _lib.pg_index_layer(self._h, i, C.byref(cnt), C.byref(R), None, None, None)
        if st != 0:
            raise PGError(st, "pg_index_layer")
        m, R = cnt.value, R.value
        dev = self.device
        gid = torch.empty(m, dtype=torch.int32, device=dev)
        nbr = torch.empty((m, R), dtype=torch.int32, device=dev)
        deg = torch.empty(m, dtype=torch.int32, device=dev)
        self.ctx._check(_lib.pg_index_export_layer(self.ctx.handle, self._h, i, _ptr(gid),
                                                   _ptr(nbr), _ptr(deg)), "pg_index_export_layer")
        return gid, nbr, deg

    def reserve(self, capacity: int):
        """Private copy of the points with room for `capacity` rows (pg_index_reserve)."""
        self.ctx._check(_lib.pg_index_reserve(self.ctx.handle, self._h, int(capacity)),
                        "pg_index_reserve")

    def insert(self, X: torch.Tensor, ef: int, upper_beam: int = 1):
        """Batched insertion of the rows of X (pg_index_insert); new ids follow n."""
        X = _dev(X, torch.float32, "X")
        self.ctx._check(_lib.pg_index_insert(self.ctx.handle, self._h, _ptr(X), X.shape[0], ef,
                                             upper_beam), "pg_index_insert")

    def quality(self):
        """(OptKCNA iterations run, sample size n_s, estimates per iteration) of
        the last build's quality examination (pg_index_quality)."""
        it, ns = C.c_int32(), C.c_int64()
        est = (C.c_double * 16)()
        _lib.pg_index_quality(self._h, C.byref(it), C.byref(ns), est)
        return it.value, ns.value, [est[i] for i in range(min(it.value, 16))]

    def phase_seconds(self):
        arr = (C.c_double * 6)()
        _lib.pg_index_phase_seconds(self._h, arr)
        return dict(zip(["knn", "prune", "union", "connect", "acquire", "layers"], list(arr)))

    def search(self, Q: torch.Tensor, k: int, beam: int, upper_beam: int = UPPER_BEAM,
               flat: bool = False, precision="fp32"):
        """k-ANN queries; upper layers use pool width upper_beam (1 = greedy)."""
        Q = _dev(Q, torch.float32, "Q")
        nq = Q.shape[0]
        ids = torch.empty((nq, k), dtype=torch.int32, device=Q.device)
        dist = torch.empty((nq, k), dtype=torch.float32, device=Q.device)
        self.ctx._check(_lib.pg_search(self.ctx.handle, self._h, _ptr(Q), nq, k, beam,
                                       upper_beam, 1 if flat else 0, PRECISION[precision],
                                       _ptr(ids), _ptr(dist)), "pg_search")
        return ids, dist

    def search_host(self, Q: np.ndarray, k: int, beam: int, upper_beam: int = UPPER_BEAM,
                    flat: bool = False, out_ids: np.ndarray | None = None,
                    out_dist: np.ndarray | None = None, precision="fp32"):
        """Host buffers in and out (copies inside the call)."""
        if not (isinstance(Q, np.ndarray) or isinstance(Q, torch.Tensor)):
            raise TypeError("Q must be a host array")
        nq = Q.shape[0]
        if out_ids is None:
            out_ids = np.empty((nq, k), np.int32)
        if out_dist is None:
            out_dist = np.empty((nq, k), np.float32)

        def hp(a):
            if isinstance(a, torch.Tensor):
                return C.c_void_p(a.data_ptr())
            return a.ctypes.data_as(C.c_void_p)

        self.ctx._check(_lib.pg_search_host(self.ctx.handle, self._h, hp(Q), nq, k, beam,
                                            upper_beam, 1 if flat else 0, PRECISION[precision],
                                            hp(out_ids), hp(out_dist)),
                        "pg_search_host")
        return out_ids, out_dist

    def close(self):
        if getattr(self, "_h", None):
            _lib.pg_index_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------- serving
def serve_simulate(kind, rows, shape, slots: int = 4, max_batch: int = 1024,
                   budget_bytes: int = 0, work_us: int = 200, bytes_per_row: int = 0):
    """The serving scheduler with simulated work on the host (pg_serve_simulate):
    per-request event positions, worker and group, and the stats."""
    kind = np.ascontiguousarray(kind, np.int32)
    rows = np.ascontiguousarray(rows, np.int32)
    shape = np.ascontiguousarray(shape, np.int32)
    n = len(kind)
    start = np.full(n, -1, np.int64)
    end = np.full(n, -1, np.int64)
    slot = np.full(n, -2, np.int32)
    group = np.full(n, -1, np.int64)
    version = np.full(n, -1, np.int64)
    st = (C.c_int64 * len(SERVE_STATS))()

    def p(a):
        return a.ctypes.data_as(C.c_void_p)

    rc = _lib.pg_serve_simulate(slots, max_batch, budget_bytes, n, p(kind), p(rows), p(shape),
                                work_us, bytes_per_row, p(start), p(end), p(slot), p(group),
                                p(version), st)
    if rc != 0:
        raise PGError(rc, "pg_serve_simulate")
    return dict(start=start, end=end, slot=slot, group=group, version=version,
                stats=dict(zip(SERVE_STATS, list(st))))


SERVE_STATS = ["batches", "requests", "queries", "inserted", "max_in_flight",
               "admission_waits"]


class Server:
    """Serving loop over a growable index (pg_serve_*): query and insertion
    requests with host buffers; query groups and insertions run on `slots`
    concurrent workers, each query group on the index version pinned when it
    was dispatched; tickets complete out of order."""

    def __init__(self, index: Index, max_batch: int = 1024, slots: int = 4):
        self.index, self.ctx = index, index.ctx
        self._h = C.c_void_p()
        self.ctx._check(_lib.pg_serve_start(self.ctx.handle, index._h, max_batch, slots,
                                            C.byref(self._h)), "pg_serve_start")
        self._keep = {}

    @staticmethod
    def _chk(st, what):
        # the context's error message belongs to the worker while serving
        if st != 0:
            raise PGError(st, what)

    def submit_query(self, Q: np.ndarray, k: int, beam: int, upper_beam: int = UPPER_BEAM):
        """Returns (ticket, ids, dist); ids/dist are filled once the ticket completes."""
        Q = np.ascontiguousarray(Q, np.float32)
        ids = np.empty((Q.shape[0], k), np.int32)
        dist = np.empty((Q.shape[0], k), np.float32)
        t = C.c_int64()
        self._chk(_lib.pg_serve_submit_query(
            self._h, Q.ctypes.data_as(C.c_void_p), Q.shape[0], k, beam, upper_beam,
            ids.ctypes.data_as(C.c_void_p), dist.ctypes.data_as(C.c_void_p), C.byref(t)),
            "pg_serve_submit_query")
        self._keep[t.value] = (Q, ids, dist)
        return t.value, ids, dist

    def submit_insert(self, X: np.ndarray, ef: int, upper_beam: int = 1) -> int:
        X = np.ascontiguousarray(X, np.float32)
        t = C.c_int64()
        self._chk(_lib.pg_serve_submit_insert(self._h, X.ctypes.data_as(C.c_void_p),
                                                    X.shape[0], ef, upper_beam, C.byref(t)),
                        "pg_serve_submit_insert")
        self._keep[t.value] = (X,)
        return t.value

    def wait(self, ticket: int, timeout_s: float = 60.0) -> bool:
        done = C.c_int32()
        self._chk(_lib.pg_serve_wait(self._h, ticket, timeout_s, C.byref(done)),
                        "pg_serve_wait")
        if done.value:
            self._keep.pop(ticket, None)
        return bool(done.value)

    def set_queue_limit(self, limit: int):
        """Refuse submissions (PGError CAPACITY) while `limit` requests are pending."""
        self._chk(_lib.pg_serve_set_queue_limit(self._h, int(limit)),
                        "pg_serve_set_queue_limit")

    def latency(self, ticket: int) -> float:
        """Seconds from submission to completion of a completed ticket."""
        v = C.c_double()
        self._chk(_lib.pg_serve_latency(self._h, ticket, C.byref(v)), "pg_serve_latency")
        return v.value

    def set_precision(self, precision: str):
        """Distance form ("fp32", "bf16", "fp8") of query requests submitted from now on."""
        self._chk(_lib.pg_serve_set_precision(self._h, PRECISION[precision]),
                  "pg_serve_set_precision")

    def set_budget(self, nbytes: int):
        """Device scratch the groups in flight may hold together (0: no limit)."""
        self._chk(_lib.pg_serve_set_budget(self._h, int(nbytes)), "pg_serve_set_budget")

    def stats(self):
        a = (C.c_int64 * len(SERVE_STATS))()
        _lib.pg_serve_stats(self._h, a, len(SERVE_STATS))
        return dict(zip(SERVE_STATS, list(a)))

    def wait_all(self, tickets, timeout_s: float = 60.0) -> bool:
        """Wait for every ticket (they complete out of order)."""
        return all(self.wait(t, timeout_s) for t in tickets)

    def stop(self):
        if getattr(self, "_h", None):
            _lib.pg_serve_stop(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass

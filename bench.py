#!/usr/bin/env python
"""Benchmark of the graph-construction path on GB300.

Workload: 1,000,000 x 128 float32 points (byte-valued Gaussian mixture of
1,024 clusters, sigma 20), squared L2, exact kNN K=64, candidate pool L=200,
degree bound R=32, alpha 66 / 60 degrees, I=2 OptKCNA iterations, NSWG
routing layers (M=16); 10,000 queries, k=10, beams 32..256.

A step is one full pg_build_rng (kNN -> 2 x [prune, reverse union, prune,
connect, self-search] -> final RNG refinement -> routing layers) over the
resident points.  value = build points/s over the whole job.  Under torchrun
every rank builds its own replica (independent problems, weak scaling, no
data-path collective); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic  # noqa: E402

SERVE_SLOTS = 4  # concurrent query groups of the serving loop
WORKLOAD = 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16"],
                    help="form of the timed build (the other form is timed once beside it)")
    ap.add_argument("--no-other-form", action="store_true")
    ap.add_argument("--n", type=int, default=None, help="shrink the workload (tests only)")
    ap.add_argument("--nq", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-queries", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-screen", action="store_true")
    ap.add_argument("--no-quality", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="fixed launch configurations (no tuning launches, for ncu captures)")
    ap.add_argument("--sweep", action="store_true",
                    help="alpha / I sweep on the workload instead of the benchmark line")
    ap.add_argument("--extra", choices=["nswg-1m-d96-cosine", "serve-2m-d384-ip"], default=None,
                    help="the NSWG cosine or the 2M x 384 serving workload instead of the "
                         "benchmark line")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
class Clocks:
    """nvidia-smi sampling of SM clocks / throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="pg_clocks_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def oracle_build_rate(D, w, ns: int, threads: int | None = None):
    """Oracle stages on the first ns points of the workload, extrapolated
    to the full n: exact kNN scaled by (n/ns)^2, every other stage by n/ns."""
    import oracle
    if threads:
        oracle.set_threads(threads)
    n = D.shape[0]
    S = np.ascontiguousarray(D[:ns])
    K, L, R = w["K"], w["L"], w["R"]
    t = {}
    t0 = time.perf_counter()
    ids, _ = oracle.knn(S, K)
    t["knn"] = time.perf_counter() - t0
    ep = oracle.medoid(S)
    off = np.arange(ns + 1, dtype=np.int64) * K
    cand = ids.ravel()
    t["prune"] = t["union"] = t["connect"] = t["acquire"] = 0.0
    for it in range(3):
        alpha = 66.0 if it < 2 else 60.0
        t0 = time.perf_counter()
        nb, dg = oracle.prune(S, off, cand, R, alpha)
        t["prune"] += time.perf_counter() - t0
        t0 = time.perf_counter()
        uo, ui = oracle.reverse_union(nb, dg)
        t["union"] += time.perf_counter() - t0
        t0 = time.perf_counter()
        nb, dg = oracle.prune(S, uo, ui, R, alpha)
        t["prune"] += time.perf_counter() - t0
        t0 = time.perf_counter()
        nb, dg, _ = oracle.connect(S, nb, dg, ep)
        t["connect"] += time.perf_counter() - t0
        if it < 2:
            t0 = time.perf_counter()
            c = oracle.acquire(S, nb, dg, L)
            t["acquire"] += time.perf_counter() - t0
            off = np.arange(ns + 1, dtype=np.int64) * L
            cand = c.ravel()
    scale = n / ns
    total = t["knn"] * scale * scale + (t["prune"] + t["union"] + t["connect"] + t["acquire"]) * scale
    sampled = sum(t.values())
    return n / total, sampled, t


def cpu_model():
    """CPU model from /proc/cpuinfo; on Arm (no model name) the implementer and
    part codes, e.g. 0x41 / 0xd4f for an Arm Neoverse V2 (NVIDIA Grace)."""
    import platform
    impl = part = None
    try:
        for line in open("/proc/cpuinfo"):
            key = line.lower()
            if key.startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
            if key.startswith("cpu implementer") and impl is None:
                impl = line.split(":", 1)[1].strip()
            if key.startswith("cpu part") and part is None:
                part = line.split(":", 1)[1].strip()
    except OSError:
        pass
    if impl or part:
        names = {("0x41", "0xd4f"): "Arm Neoverse V2"}
        return f"{platform.machine()} implementer {impl} part {part}" + (
            f" ({names[(impl, part)]})" if (impl, part) in names else "")
    return platform.machine() or "unknown"


# ------------------------------------------------------------------ arms
def job_rate(ms_local: float, n_per_rank: int, world: int, device: str = "cpu"):
    """Whole-job rate of independent replicas (weak scaling): every rank builds
    its own n-point index; the step time is the slowest rank's (max over
    ranks), and the job processes world * n points per step.  Returns
    (ms_max, points_per_s).  Needs an initialised process group when world > 1."""
    ms = ms_local
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * n_per_rank / (ms / 1e3)


def serving_measure(pg, idx, Q, X, ins, k, beam, upper_beam, seed=7):
    """The serving loop on a built index (groups of up to 1,024 queries on
    SERVE_SLOTS workers, host buffers), request sizes drawn from {1, 8, 32,
    128, 1024} queries, two insertion batches of `ins` points of X after
    requests 100 and 200 of 300:
      saturated: all 300 requests queued at once, with SERVE_SLOTS workers,
      with one, and with SERVE_SLOTS workers and FP8-screened queries, for
      requests/s and queries/s;
      poisson: the same mix arriving as a Poisson process at 70% of the
      saturated request rate, for the latency of each request from
      submission to completion (p50 / p99, host clock);
    then 200 single-query requests one at a time.  The index must have room
    for 8 ins more points."""
    Qh = np.asarray(Q)
    nq = len(Qh)
    rs = np.random.default_rng(seed)
    sizes = rs.choice([1, 8, 32, 128, 1024], size=300)
    cursor = {"q": 0, "x": 0}

    def run_stream(srv, gaps=None):
        tickets, queries, nqs = [], [], 0
        t0 = time.perf_counter()
        for r, sz in enumerate(sizes):
            if gaps is not None:
                due = t0 + gaps[r]
                while True:
                    left = due - time.perf_counter()
                    if left <= 0:
                        break
                    time.sleep(left if left > 1e-3 else 0)
            if r in (100, 200):
                j = cursor["x"]
                cursor["x"] += 1
                tickets.append(srv.submit_insert(X[j * ins:(j + 1) * ins], 64, upper_beam))
            rows = (cursor["q"] + np.arange(int(sz))) % nq
            cursor["q"] += int(sz)
            nqs += int(sz)
            t, _, _ = srv.submit_query(Qh[rows], k, beam, upper_beam)
            tickets.append(t)
            queries.append(t)
        assert srv.wait_all(tickets, 600.0)
        secs = time.perf_counter() - t0
        lat = [srv.latency(t) * 1e3 for t in queries]
        return secs, nqs, lat

    sat = {}
    for slots, prec in ((SERVE_SLOTS, "fp32"), (1, "fp32"), (SERVE_SLOTS, "fp8")):
        srv = pg.Server(idx, max_batch=1024, slots=slots)
        srv.set_precision(prec)
        secs, nqs, _ = run_stream(srv)
        st = srv.stats()
        srv.stop()
        sat[(slots, prec)] = {"seconds": secs, "requests_per_s": len(sizes) / secs,
                              "queries_per_s": nqs / secs, "groups": int(st["batches"]),
                              "max_in_flight": int(st["max_in_flight"])}
    rate = 0.7 * sat[(SERVE_SLOTS, "fp32")]["requests_per_s"]
    gaps = np.cumsum(rs.exponential(1.0 / rate, size=len(sizes)))
    srv = pg.Server(idx, max_batch=1024, slots=SERVE_SLOTS)
    secs, nqs, lat = run_stream(srv, gaps)
    st = srv.stats()
    single = []
    for i in range(200):
        t1 = time.perf_counter()
        tk, _, _ = srv.submit_query(Qh[i % nq:i % nq + 1], k, beam, upper_beam)
        srv.wait(tk, 60.0)
        single.append((time.perf_counter() - t1) * 1e3)
    srv.stop()
    return {"slots": SERVE_SLOTS, "requests": len(sizes), "queries": int(sizes.sum()),
            "inserted_per_stream": 2 * ins,
            "saturated": sat[(SERVE_SLOTS, "fp32")],
            "saturated_one_worker": sat[(1, "fp32")],
            "saturated_fp8_screen": sat[(SERVE_SLOTS, "fp8")],
            "poisson": {"rate_requests_per_s": rate, "seconds": secs,
                        "queries_per_s": nqs / secs, "groups": int(st["batches"]),
                        "max_in_flight": int(st["max_in_flight"]),
                        "admission_waits": int(st["admission_waits"]),
                        "p50_ms": float(np.percentile(lat, 50)),
                        "p99_ms": float(np.percentile(lat, 99))},
            "single_query_p50_ms": float(np.percentile(single, 50)),
            "single_query_p99_ms": float(np.percentile(single, 99)),
            "stream": f"300 query requests of 1/8/32/128/1024 queries (k={k}, beam {beam}) "
                      f"with two insertion batches of {ins} points, host buffers"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    n = args.n or synthetic.WORKLOADS[WORKLOAD]["n"]
    D, _, w = synthetic.workload(WORKLOAD, n=n, nq=1)
    ns = min(n, 8000)
    cores = oracle.num_threads()
    vals = []
    for i in range(args.warmup + args.steps):
        v, sampled, _ = oracle_build_rate(D, w, ns)
        if i >= args.warmup:
            vals.append(v)
    value = statistics.mean(vals)
    sample = (f"oracle stages (exact kNN, 3x[prune, reverse union, prune, connect], 2x self-search) "
              f"on the first {ns} points of the {n}x{w['d']} workload; kNN time scaled by "
              f"(n/{ns})^2, other stages by n/{ns}")
    line = {
        "impl": "reference", "metric": "build_points_per_s", "value": value,
        "unit": "points/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": n / value * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"], "n": n, "d": w["d"], "K": w["K"], "L": w["L"],
                   "R": w["R"], "iters": 2},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle",
                         "sample": sample, "cpu": cpu_model()},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2410_01231_gb300 as pg

    n = args.n or synthetic.WORKLOADS[WORKLOAD]["n"]
    nq = args.nq or synthetic.WORKLOADS[WORKLOAD]["nq"]
    D, Q, w = synthetic.workload(WORKLOAD, n=n, nq=nq)
    params = dict(K=w["K"], L=w["L"], R=w["R"], M=16, alpha_deg=66.0, alpha_final_deg=60.0,
                  iters=2, precision=args.precision, route_layers=1, seed=0)
    Dd = torch.from_numpy(D).cuda()
    Qd = torch.from_numpy(Q).cuda()
    stream = torch.cuda.current_stream()
    ctx = pg.Context(stream)
    # launch configurations of the persistent kernels chosen by timing on
    # the first (warm-up) build; the timed builds use the tuned table
    ctx.set_autotune(not args.no_autotune)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    gpu_id = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            gpu_id = int(vis.split(",")[local])
        except ValueError:
            pass

    def timed_builds(prm, warmup, steps, clocks=None):
        """warmup untimed builds, then `steps` builds bracketed by a barrier and
        a synchronize on both sides and timed with CUDA events on the
        context's stream; per-kernel CUDA-event times and the kernels' own
        work counters over the timed builds."""
        for _ in range(warmup):
            pg.Index.build_rng(ctx, Dd, **prm).close()
        ctx.set_timing(True)
        launches0 = ctx.launches
        barrier()
        if clocks:
            clocks.start()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        nvtx = getattr(torch.cuda, "nvtx", None)
        try:  # names the timed region for profilers (ncu --nvtx-include timed/)
            nvtx.range_push("timed")
        except Exception:
            nvtx = None
        ev0.record(stream)
        phases = []
        for _ in range(steps):
            idx = pg.Index.build_rng(ctx, Dd, **prm)
            phases.append(idx.phase_seconds())
            idx.close()
        ev1.record(stream)
        if nvtx is not None:
            nvtx.range_pop()
        barrier()
        clk = clocks.stop() if clocks else None
        r = {"ms": ev0.elapsed_time(ev1) / steps, "launches": ctx.launches - launches0,
             "clocks": clk, "steps": steps, "warmup": warmup,
             "kt": {k: ctx.kernel_time(k) for k in ("knn", "prune", "union", "connect", "search",
                                                    "medoid")},
             "knn_work": ctx.kernel_work("knn"),
             "work": {c: ctx.counter(c) for c in ("search_expansions", "search_evaluations",
                                                  "search_bytes", "prune_rows",
                                                  "prune_candidates", "prune_bytes")},
             "conn_edges": ctx.counter("connect_edges"),
             "conn_full": ctx.counter("connect_full_rounds"),
             "phases": ({k: statistics.mean(p[k] for p in phases) for k in phases[0]}
                        if phases else {})}
        ctx.set_timing(False)
        return r

    main_run = timed_builds(params, args.warmup, args.steps, Clocks(gpu_id))
    ms, value = job_rate(main_run["ms"], n, world, "cuda")
    kt, work = main_run["kt"], main_run["work"]
    launches, clk, phases_mean = main_run["launches"], main_run["clocks"], main_run["phases"]

    # ---------------------------------------------------------- queries
    qres = {}
    if not args.no_queries:
        idx = pg.Index.build_rng(ctx, Dd, **params)
        gt_i, gt_d = pg.knn_query(ctx, Dd, Qd, w["k"])
        kth = gt_d[:, w["k"] - 1].clone()

        def recall(ids):
            dq = ((Qd[:, None, :] - Dd[ids.long().clamp(min=0)]) ** 2).sum(-1)
            ok = (dq <= kth[:, None]) & (ids >= 0)
            return float(ok.sum(1).clamp(max=w["k"]).float().mean() / w["k"])

        curve = []
        for beam in w["beams"]:
            idx.search(Qd, w["k"], beam)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ids, _ = idx.search(Qd, w["k"], beam)
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            flat, _ = idx.search(Qd, w["k"], beam, flat=True)
            curve.append({"beam": beam, "recall": recall(ids), "qps": nq / t,
                          "recall_flat_entry": recall(flat)})
        ok = [c for c in curve if c["recall"] >= 0.95]
        best = ok[0] if ok else curve[-1]
        # FP8-screened queries (E4M3 rows, FP32 re-measure of the final pool)
        fp8 = []
        for beam in w["beams"]:
            idx.search(Qd, w["k"], beam, precision="fp8")
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ids, _ = idx.search(Qd, w["k"], beam, precision="fp8")
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            fp8.append({"beam": beam, "recall": recall(ids), "qps": nq / t})
        lat = []
        for i in range(min(200, nq)):
            t0 = time.perf_counter()
            idx.search(Qd[i:i + 1], w["k"], best["beam"])
            lat.append((time.perf_counter() - t0) * 1e3)
        qres = {"curve": curve, "fp8_screen_curve": fp8,
                "beam_at_0.95": best["beam"] if ok else None,
                "recall": best["recall"], "qps": best["qps"],
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "latency": "single-query requests, host wall time per call incl. launch + sync"}
        idx.close()

    # ---------------------------------------------------------- serving
    # The serving loop on the index just measured (groups of up to 1,024
    # queries on four workers, host buffers), request sizes drawn from
    # {1, 8, 32, 128, 1024} queries (k = 10, beam 48, upper_beam 16), two
    # insertion batches of 1% of n after requests 100 and 200 of 300:
    #   saturated: all 300 requests queued at once, with four workers, with
    #   one, and with four workers and FP8-screened queries, for requests/s
    #   and queries/s;
    #   poisson: the same mix arriving as a Poisson process at 70% of the
    #   four-worker saturated request rate, for the latency of each request
    #   from submission to completion (p50 / p99, host clock);
    # then 200 single-query requests one at a time.
    serve = {}
    if not args.no_serve:
        ins = max(100, n // 100)
        X = synthetic.inserts(WORKLOAD, 8 * ins)
        idx = pg.Index.build_rng(ctx, Dd, **params)
        idx.reserve(n + 8 * ins)
        barrier()
        serve = serving_measure(pg, idx, Q, X, ins, w["k"], 48, 16)
        idx.close()

    # ------------------------------------- the 960-d real-valued workload
    # The 1M x 960 real-valued recipe (512 centres U[0,1]^960, sigma 0.1)
    # sampled at 100,000 points with the same cluster density (51 clusters):
    # the kNN graph (K = 64) in the FP32 form and in the certified screened
    # form (hi/lo BF16 tiles, FP32 re-measure, FP64 near ties, FP32 tiles for
    # rows the bound cannot certify), then the whole RNG build in both forms
    # (edge agreement) and recall@10 of 1,000 queries against exact kNN.
    screen = {}
    if not args.no_screen:
        w3 = synthetic.WORKLOADS[3]
        ns = min(100_000, max(20_000, n // 10))
        ncl = max(8, w3["clusters"] * ns // w3["n"])
        X3, c3 = synthetic.mixture_float(ns, w3["d"], ncl, 1234 + 3)
        Q3, _ = synthetic.mixture_float(1000, w3["d"], ncl, 5678 + 3, centres=c3)
        X3d, Q3d = torch.from_numpy(X3).cuda(), torch.from_numpy(Q3).cuda()
        times, lists = {}, {}
        for prec in ("fp32", "bf16"):
            pg.build_knn(ctx, X3d, w3["K"], precision=prec)  # warm-up
            barrier()
            ctx.set_timing(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ids3, ds3 = pg.build_knn(ctx, X3d, w3["K"], precision=prec)
            e1.record(stream)
            barrier()
            times[prec] = e0.elapsed_time(e1)
            lists[prec] = (ids3, ds3)
            if prec == "bf16":
                fallback = ctx.counter("knn_fallback_rows")
                tiles_ms, _ = ctx.kernel_time("knn")
                tiles_flops = ctx.kernel_work("knn")
            ctx.set_timing(False)
        same_lists = bool(torch.equal(lists["fp32"][0], lists["bf16"][0]) and
                          torch.equal(lists["fp32"][1], lists["bf16"][1]))
        del lists
        # iterations at alpha 60: at 66 every reached node of these tight 960-d
        # clusters is full, and connectivity goes through edge replacement,
        # whose rounds run one at a time (about 95 s at this size)
        p3 = dict(K=w3["K"], L=w3["L"], R=w3["R"], M=16, alpha_deg=60.0, alpha_final_deg=60.0,
                  iters=2, route_layers=1, seed=0)
        builds, graphs, phases3 = {}, {}, {}
        gt_i, gt_d = pg.knn_query(ctx, X3d, Q3d, 10)
        kth3 = gt_d[:, 9].clone()
        for prec in ("fp32", "bf16"):
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            idx3 = pg.Index.build_rng(ctx, X3d, precision=prec, **p3)
            e1.record(stream)
            barrier()
            builds[prec] = e0.elapsed_time(e1)
            phases3[prec] = idx3.phase_seconds()
            _, nb3, dg3 = idx3.layer(0)
            graphs[prec] = (nb3.clone(), dg3.clone())
            if prec == "bf16":
                curve3 = []
                for beam in w3["beams"]:
                    ids, _ = idx3.search(Q3d, 10, beam)
                    dq = ((Q3d[:, None, :] - X3d[ids.long().clamp(min=0)]) ** 2).sum(-1)
                    ok = (dq <= kth3[:, None] * (1 + 1e-6)) & (ids >= 0)
                    curve3.append({"beam": beam,
                                   "recall_at_10": float(ok.sum(1).clamp(max=10).float().mean()
                                                         / 10)})
            idx3.close()
        a, b = graphs["fp32"], graphs["bf16"]
        same_rows = int(((a[0] == b[0]).all(1) & (a[1] == b[1])).sum())
        screen = {"workload": f"{w3['name']} recipe at n={ns} ({ncl} clusters)", "K": w3["K"],
                  "build_params": "K 64, L 200, R 32, alpha 60 / 60, I = 2, routing layers",
                  "knn_fp32_ms": times["fp32"], "knn_bf16_screen_ms": times["bf16"],
                  "knn_speedup": times["fp32"] / times["bf16"],
                  "knn_lists_identical": same_lists,
                  "screen_fallback_rows": fallback,
                  "screen_tiles_ms": tiles_ms,
                  "screen_tiles_tflops": tiles_flops / (tiles_ms / 1e3) / 1e12 if tiles_ms else None,
                  "screen_tiles_note": "executed contraction: 2 n^2 x 3d (hi.hi + hi.lo + lo.hi)",
                  "build_fp32_ms": builds["fp32"], "build_bf16_screen_ms": builds["bf16"],
                  "build_phase_s": phases3,
                  "edge_agreement_rows": same_rows / ns, "graphs_identical": same_rows == ns,
                  "queries": curve3}
        del X3d, Q3d, graphs

    # ------------------------------------------------ the other precision form
    # Timed like the main form (CUDA events on the context's stream, barrier
    # and synchronize on both sides) over min(steps, 3) builds after one
    # warm-up: the FP32 form takes several seconds per build.
    forms = {args.precision: {"ms_per_build": ms, "points_per_s": value, "steps": args.steps,
                              "kernel_ms_per_build": {k: v[0] / args.steps
                                                      for k, v in kt.items()}}}
    identical = None
    other_run = None
    fp32_peak = ctx.measure_fp32_peak()
    if not args.no_other_form:
        other = "fp32" if args.precision == "bf16" else "bf16"
        p2 = dict(params, precision=other)
        other_run = timed_builds(p2, 1, min(args.steps, 3))
        forms[other] = {"ms_per_build": other_run["ms"],
                        "points_per_s": n / (other_run["ms"] / 1e3),
                        "steps": other_run["steps"], "warmup": other_run["warmup"],
                        "kernel_ms_per_build": {k: v[0] / other_run["steps"]
                                                for k, v in other_run["kt"].items()},
                        "phase_s": other_run["phases"]}
        a = pg.Index.build_rng(ctx, Dd, **params)
        b = pg.Index.build_rng(ctx, Dd, **p2)
        _, na, da = a.layer(0)
        _, nb_, db = b.layer(0)
        identical = bool(torch.equal(na, nb_) and torch.equal(da, db))
        a.close()
        b.close()

    # ------------------------------------------- quality examination
    # One more (untimed) build with the quality examination of Section 5.2 on
    # (Theorem 3's sample, eps 0.6, recall of the first K entries of C(u)):
    # the loop of Algorithm 6 stops once the sampled k-CNA recall reaches the
    # target, at most `iters` iterations; the iterations it chose and its
    # estimates after each are reported.
    quality = None
    if not args.no_quality:
        target = 0.99
        qb = pg.Index.build_rng(ctx, Dd, **dict(params, quality_target=target, quality_eps=0.6))
        it_run, ns, est = qb.quality()
        qb.close()
        quality = {"target": target, "eps": 0.6, "sample_size": ns, "iterations_run": it_run,
                   "iterations_max": params["iters"], "estimates": est,
                   "note": "k-CNA recall of the first K entries of C(u) on the Theorem 3 sample"}

    # --------------------------------------------------------- tie budget
    # One more (untimed) build of the main form with the pruning kernels'
    # tie accounting on: decisions of the occlusion test whose relative
    # margin is below 1e-5, the FP64 rechecks and the rechecks whose FP64
    # outcome differed from plain FP32, over all six pruning calls.
    ctx.set_timing(True)  # resets the device counters
    ctx.set_tie_count(True)
    pg.Index.build_rng(ctx, Dd, **params).close()
    tie = {k: ctx.counter("prune_" + k) for k in ("edges", "near_ties", "fp64_rechecks",
                                                   "fp64_flips")}
    ctx.set_tie_count(False)
    ctx.set_timing(False)
    tie["near_tie_share_of_edges"] = tie["near_ties"] / max(1, tie["edges"])
    tie["note"] = ("counts over the six pruning calls of one build (base layer); every near-tie "
                   "decision is decided exactly (integer distances or the FP64 recheck), so the "
                   "allowed mismatches are 0; mismatches against the oracle: oracle_check")

    # ------------------------------------------------------------- e2e
    # The same build through the C ABI with HOST buffers (pg_build_rng_host):
    # the pinned host points are uploaded, the graph is built and the base
    # graph (nbr [n][R], deg [n]) is read back inside the call; wall time of
    # the call, averaged over min(steps, 3) calls after one warm-up.
    e2e = None
    if not args.no_e2e:
        Dh = torch.from_numpy(D).pin_memory()
        nbr_h = torch.empty((n, w["R"]), dtype=torch.int32).pin_memory()
        deg_h = torch.empty(n, dtype=torch.int32).pin_memory()
        pg.Index.build_rng_host(ctx, Dh, nbr_h, deg_h, **params)
        reps = min(args.steps, 3)
        barrier()
        t0 = time.perf_counter()
        for _ in range(reps):
            pg.Index.build_rng_host(ctx, Dh, nbr_h, deg_h, **params)
        barrier()
        t = (time.perf_counter() - t0) / reps
        e2e = {"value": world * n / t, "unit": "points/s", "seconds_per_build": t,
               "calls": reps, "api": "pg_build_rng_host (host buffers, pinned)",
               "h2d_bytes_per_step": int(D.nbytes),
               "d2h_bytes_per_step": int(nbr_h.numel() * 4 + deg_h.numel() * 4)}

    # -------------------------------------------------------- roofline
    # Every figure is algorithmic work over the summed CUDA-event time of the
    # kernel's launches inside the timed region (base graph and routing
    # layers).  kNN: 2 d flops per (row, point) pair.  Beam search: one data
    # row per distance evaluation plus one R-entry adjacency row per
    # expansion.  Prune: one data row plus (id, distance) per examined
    # candidate, plus the point's own row.  A data row is 4d bytes, d bytes
    # where the screened form gathers byte rows (counted by the kernels).
    # Kernels timed inside a seconds-long build take the sustained peaks.
    pk = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    pk_sms = torch.cuda.get_device_properties(0).multi_processor_count

    def rooflines_of(run, form):
        out = {}
        steps = run["steps"]
        knn_ms = run["kt"]["knn"][0]
        if knn_ms > 0:
            a = run["knn_work"] / (knn_ms / 1e3) / 1e12
            if form == "fp32":
                out["knn"] = {
                    "kernel": "k_knn_fp32", "bound": "alu", "achieved": a, "peak": fp32_peak,
                    "unit": "TFLOP/s", "frac": a / fp32_peak if fp32_peak else None,
                    "traffic": None,
                    "peak_source": "measured FP32 FMA throughput (pg_measure_fp32_peak, this run)"}
            else:
                peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1700.0))
                out["knn"] = {
                    "kernel": "k_knn_tc", "bound": "tensor", "achieved": a, "peak": peak,
                    "unit": "TFLOP/s", "frac": a / peak, "traffic": None,
                    "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)",
                    "frac_of_burst": a / pk.get("bf16_tflops", peak)}
        for name, kern, key in (("search", "k_search", "search_bytes"),
                                ("prune", "k_prune", "prune_bytes")):
            t_ms = run["kt"][name][0]
            if t_ms > 0:
                b = run["work"][key]
                a = b / (t_ms / 1e3) / 1e9
                out[name] = {
                    "kernel": kern, "bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s",
                    "frac": a / hbm, "traffic": None, "algorithmic_bytes_per_step": b / steps,
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
        if "search" in out:
            out["search"]["evaluations_per_step"] = run["work"]["search_evaluations"] / steps
        # DRAM traffic of a kernel's main launch from an ncu capture recorded
        # in profiles/roofline_traffic.json, valid only while the kernel's
        # source file is byte-identical to the one captured (else null)
        try:
            import hashlib
            with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
                rec = json.load(f)
            for r in out.values():
                ent = rec.get(r["kernel"])
                if not ent or ent.get("n") != n:
                    continue
                with open(os.path.join(ROOT, ent["source"]), "rb") as f:
                    if hashlib.sha256(f.read()).hexdigest() == ent["source_sha256"]:
                        # per launch where `achieved` is one launch's, per step
                        # where it is summed over the step's launches
                        r["traffic"] = ent.get("dram_bytes_per_launch",
                                               ent.get("dram_bytes_per_step"))
                        r["traffic_per"] = "launch" if "dram_bytes_per_launch" in ent else "step"
                        r["traffic_note"] = ent["note"]
                        # issue-bound kernels: the step's warp instructions (ncu)
                        # against the issue rate of every SM sub-partition at
                        # the clock sampled in the timed region
                        w = ent.get("warp_instructions_per_step")
                        name = {"k_search": "search", "k_prune": "prune"}.get(r["kernel"])
                        mhz = (run.get("clocks") or {}).get("sm_mhz")
                        if w and name and mhz:
                            t_s = run["kt"][name][0] / steps / 1e3
                            unit, per = (("evaluation", run["work"]["search_evaluations"])
                                         if name == "search" else
                                         ("candidate", run["work"]["prune_candidates"]))
                            r["issue"] = {
                                "warp_instructions_per_step": w,
                                f"warp_instructions_per_{unit}": w / (per / steps) if per else None,
                                "issue_rate_frac": w / (t_s * 4 * pk_sms * mhz * 1e6),
                                "note": ("warp instructions from the same ncu capture; the peak is "
                                         "one warp instruction per cycle per SM sub-partition")}
        except (OSError, ValueError, KeyError):
            pass
        return out

    rooflines = rooflines_of(main_run, args.precision)
    if other_run is not None:
        forms[other]["rooflines"] = rooflines_of(other_run, other)
    forms[args.precision]["rooflines"] = rooflines
    # the dominant single kernel of the step (connect is a chain of kernels)
    top = max(rooflines, key=lambda k: kt[k][0]) if rooflines else None
    roof = dict(rooflines[top], share_of_step=kt[top][0] / args.steps / ms) if top else None

    cpu = None
    oracle_check = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        ns = min(n, 40000)
        v, sampled, _ = oracle_build_rate(D, w, ns)
        cpu = {"value": v, "unit": "points/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": (f"oracle stages on the first {ns} points ({sampled:.1f} s of CPU work); "
                          f"kNN scaled by (n/ns)^2, other stages by n/ns"),
               "cpu": cpu_model()}
        # Full-size exactness of one pruning pass (untimed): the first
        # iteration's pass over the GPU's own kNN rows (alpha 66, all n rows),
        # every row against the oracle given the same candidates.
        K = w["K"]
        gi, _ = pg.build_knn(ctx, Dd, K, precision=args.precision)
        off = torch.arange(n + 1, dtype=torch.int64, device="cuda") * K
        gn, gdg = pg.prune(ctx, Dd, off, gi.reshape(-1), w["R"], 66.0, precision=args.precision)
        t0 = time.perf_counter()
        on, odg = oracle.prune(D, off.cpu().numpy(), gi.cpu().numpy().ravel(), w["R"], 66.0)
        secs = time.perf_counter() - t0
        gnh, gdh = gn.cpu().numpy(), gdg.cpu().numpy()
        bad = int(((gnh != on).any(1) | (gdh != odg)).sum())
        oracle_check = {"step": "pruning pass 1 of iteration 1 (alpha 66) on the GPU's kNN rows",
                        "rows": n, "mismatched_rows": bad,
                        "mismatched_edges": int(np.abs(gdh.astype(np.int64) - odg).sum()
                                                + (gnh != on).sum()),
                        "oracle_seconds": secs, "cores": oracle.num_threads()}
        del gi, gn, gdg
    tie["oracle_check"] = oracle_check

    line = {
        "metric": "build_points_per_s", "value": value, "unit": "points/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "bf16", "data": "synthetic",
        "config": {"workload": w["name"], "n": n, "d": w["d"], "K": w["K"], "L": w["L"],
                   "R": w["R"], "alpha": [66.0, 60.0], "iters": 2, "route_layers_M": 16,
                   "nq": nq, "k": w["k"], "precision": args.precision,
                   "index": ("RNG base graph (Algorithm 6) + NSWG routing layers (M 16) for query "
                             "entry, upper_beam 16; recall_flat_entry = medoid entry only"),
                   "query_index_form": (f"{args.precision} form (its graph equals the other "
                                        "form's: forms_identical_graph)"),
                   "l2": (f"inputs larger than L2 ({D.nbytes >> 20} MB points)" if D.nbytes > 129e6
                          else f"inputs smaller than L2 ({D.nbytes >> 20} MB points; test size)"),
                   "parallelism": "replicas"},
        "forms": forms, "forms_identical_graph": identical, "tie_budget": tie,
        "quality_examination": quality,
        "queries": qres, "serving": serve, "real_rows_d960": screen, "phase_s": phases_mean,
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in kt.items()},
        "kernel_launches_per_step": {k: v[1] / args.steps for k, v in kt.items()},
        "connect_edges_per_step": main_run["conn_edges"] / args.steps,
        "connect_full_rounds_per_step": main_run["conn_full"] / args.steps,
        "fp32_simt_peak_tflops_measured": fp32_peak,
        "autotune": {"table": pg.autotune_report().strip().splitlines(),
                     "note": ("chosen on the first warm-up build of each form; the timed builds "
                              "use the choice; numbers are ms per candidate launch")},
        "roofline": roof, "rooflines": rooflines, "clocks": clk, "gpu_launches": launches,
        "e2e": e2e, "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_sweep(args):
    """alpha and I sweeps on the 1M x 128 workload (analogues of Exp. 1-b and
    Exp. 1-a), printed as one JSON line.

    alpha (Exp. 1-b, k-CNA quality and efficiency): from the exact kNN graph,
    one OptKCNA iteration at alpha (prune, reverse union, prune, connect, then
    the k-CNA self-search of every point); the searches' throughput (points/s,
    CUDA events), the mean out-degree of the pruned graph, and the recall of
    the first 10 and K entries of C(u) on a 10,000-point sample (r(u) of
    Section 5.2, pg_kcna_recall).
    I (Exp. 1-a): full builds with I = 0..4 (alpha 66 / 60), build time and
    query recall@10 / queries/s at beams 32, 48, 64 (routing layers on)."""
    import torch
    import paper_2410_01231_gb300 as pg

    torch.cuda.set_device(0)
    n = args.n or synthetic.WORKLOADS[WORKLOAD]["n"]
    nq = args.nq or synthetic.WORKLOADS[WORKLOAD]["nq"]
    D, Q, w = synthetic.workload(WORKLOAD, n=n, nq=nq)
    K, L, R = w["K"], w["L"], w["R"]
    Dd, Qd = torch.from_numpy(D).cuda(), torch.from_numpy(Q).cuda()
    stream = torch.cuda.current_stream()
    ctx = pg.Context(stream)
    prec = args.precision

    def events():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    knn, _ = pg.build_knn(ctx, Dd, K, precision=prec)
    ep = pg.medoid(ctx, Dd)
    off = torch.arange(n + 1, dtype=torch.int64, device="cuda") * K
    sample = torch.from_numpy(pg.quality_sample(n, min(n, 10_000), 3)).cuda()
    alphas = []
    for alpha in (60.0, 62.0, 64.0, 66.0, 68.0, 70.0, 75.0):
        n1, d1 = pg.prune(ctx, Dd, off, knn.reshape(-1), R, alpha, precision=prec)
        uo, ui = pg.reverse_union(ctx, n1, d1)
        n2, d2 = pg.prune(ctx, Dd, uo, ui, R, alpha, precision=prec)
        deg_pruned = float(d2.float().mean())
        # connectivity with edge replacement: at large alpha every reached
        # node is full and the plain step has no free slot to link from
        added, replaced = pg.connect_replace(ctx, Dd, n2, d2, ep)
        pg.acquire_candidates(ctx, Dd, n2, d2, L, precision=prec)  # warm-up
        e0, e1 = events()
        e0.record(stream)
        cand = pg.acquire_candidates(ctx, Dd, n2, d2, L, precision=prec)
        e1.record(stream)
        torch.cuda.synchronize()
        secs = e0.elapsed_time(e1) / 1e3
        _, r10 = pg.kcna_recall(ctx, Dd, cand, 10, sample)
        _, rK = pg.kcna_recall(ctx, Dd, cand, K, sample)
        alphas.append({"alpha": alpha, "kcna_points_per_s": n / secs,
                       "mean_out_degree": deg_pruned, "connect_edges": added,
                       "connect_replaced_edges": replaced,
                       "kcna_recall_at_10": r10, f"kcna_recall_at_{K}": rK})
    iters = []
    for it in range(5):
        prm = dict(K=K, L=L, R=R, M=16, alpha_deg=66.0, alpha_final_deg=60.0, iters=it,
                   precision=prec, route_layers=1, seed=0)
        pg.Index.build_rng(ctx, Dd, **prm).close()
        e0, e1 = events()
        e0.record(stream)
        idx = pg.Index.build_rng(ctx, Dd, **prm)
        e1.record(stream)
        torch.cuda.synchronize()
        build_s = e0.elapsed_time(e1) / 1e3
        gt_i, gt_d = pg.knn_query(ctx, Dd, Qd, w["k"])
        kth = gt_d[:, w["k"] - 1].clone()
        curve = []
        for beam in (32, 48, 64):
            idx.search(Qd, w["k"], beam)
            e0, e1 = events()
            e0.record(stream)
            ids, _ = idx.search(Qd, w["k"], beam)
            e1.record(stream)
            torch.cuda.synchronize()
            dq = ((Qd[:, None, :] - Dd[ids.long().clamp(min=0)]) ** 2).sum(-1)
            ok = (dq <= kth[:, None]) & (ids >= 0)
            rec = float(ok.sum(1).clamp(max=w["k"]).float().mean() / w["k"])
            curve.append({"beam": beam, "recall_at_10": rec,
                          "qps": nq / (e0.elapsed_time(e1) / 1e3)})
        _, nb, dg = idx.layer(0)
        iters.append({"iters": it, "build_s": build_s, "points_per_s": n / build_s,
                      "mean_out_degree": float(dg.float().mean()), "queries": curve})
        idx.close()
    # initial KNNG (Exp. 12): 2-hop refinement from a random draw with t
    # iterations against the exact tiles, kNN recall@K on the 10,000-point
    # sample, then the full build from it and its queries at beam 48
    inits = []
    for t in (-1, 0, 2, 4, 8):
        e0, e1 = events()
        e0.record(stream)
        if t < 0:
            gi, _ = pg.build_knn(ctx, Dd, K, precision=prec)
        else:
            gi, _, upd = pg.knn_descent(ctx, Dd, K, t, seed=0)
        e1.record(stream)
        torch.cuda.synchronize()
        knn_s = e0.elapsed_time(e1) / 1e3
        _, rK = pg.kcna_recall(ctx, Dd, gi, K, sample)
        del gi
        prm = dict(K=K, L=L, R=R, M=16, alpha_deg=66.0, alpha_final_deg=60.0, iters=2,
                   precision=prec, route_layers=1, seed=0, knn_descent_iters=t)
        e0, e1 = events()
        e0.record(stream)
        idx = pg.Index.build_rng(ctx, Dd, **prm)
        e1.record(stream)
        torch.cuda.synchronize()
        build_s = e0.elapsed_time(e1) / 1e3
        ids, _ = idx.search(Qd, w["k"], 48)
        gt_i, gt_d = pg.knn_query(ctx, Dd, Qd, w["k"])
        kth = gt_d[:, w["k"] - 1]
        dq = ((Qd[:, None, :] - Dd[ids.long().clamp(min=0)]) ** 2).sum(-1)
        ok = (dq <= kth[:, None]) & (ids >= 0)
        rec = float(ok.sum(1).clamp(max=w["k"]).float().mean() / w["k"])
        idx.close()
        inits.append({"init": "exact tiles" if t < 0 else f"2-hop x{t}", "knn_s": knn_s,
                      f"knn_recall_at_{K}": rK, "build_s": build_s,
                      "query_recall_at_10_beam48": rec})
    print(json.dumps({"sweep": "alpha (one OptKCNA iteration from the kNN graph), I (full "
                               "builds), initial KNNG", "workload": w["name"], "n": n,
                      "d": w["d"], "K": K, "L": L, "R": R, "precision": prec, "alpha": alphas,
                      "iters": iters, "init": inits}), flush=True)


def run_extra(args):
    """One of the two other single-GPU workloads, printed as one JSON line:
    nswg-1m-d96-cosine (unit Gaussian rows, NSWG, Algorithm 7) or
    serve-2m-d384-ip (4,096-cluster sphere mixture, inner product, NSWG, then
    the serving stream with insertions).  The NSWG build in the screened form
    (K 64, L 200, R 32, M 16, I 2, alpha 66 / 60 for the cosine workload and
    60 / 60 for the serving workload, edge replacement on) timed
    with CUDA events after one warm-up build (none at 2M), with its phases,
    layer sizes and the mean out-degree of layer 0; recall@10 against the
    exact kNN of the queries (the library's FP32 tiles) and queries/s per
    beam, FP32 and FP8-screened queries.  For the cosine workload also the
    build with a final angle of 70 and 80 degrees (its out-degree and
    recall), for the serving workload the serving stream of the benchmark
    line on that index.  Clocks are sampled during the timed build."""
    import torch
    import paper_2410_01231_gb300 as pg

    c = {"nswg-1m-d96-cosine": 4, "serve-2m-d384-ip": 5}[args.extra]
    torch.cuda.set_device(0)
    D, Q, w = synthetic.workload(c, n=args.n, nq=args.nq)
    n, nq, k = w["n"], w["nq"], w["k"]
    Dd, Qd = torch.from_numpy(D).cuda(), torch.from_numpy(Q).cuda()
    stream = torch.cuda.current_stream()
    ctx = pg.Context(stream)
    ctx.set_autotune(not args.no_autotune)
    # the serving workload's 4,096 tight clusters leave every reached node
    # full at 66 degrees, so its iterations take 60 (as the 960-d sample)
    alpha_it = 66.0 if c == 4 else 60.0
    base = dict(metric=w["metric"], K=w["K"], L=w["L"], R=w["R"], M=w["M"], alpha_deg=alpha_it,
                alpha_final_deg=60.0, iters=2, precision="bf16", seed=0)

    def events():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed_build(prm, warm, clocks=None):
        for _ in range(warm):
            pg.Index.build_nswg(ctx, Dd, **prm).close()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        e0, e1 = events()
        e0.record(stream)
        idx = pg.Index.build_nswg(ctx, Dd, **prm)
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop() if clocks else None
        return idx, e0.elapsed_time(e1) / 1e3, clk

    gt_i, gt_d = pg.knn_query(ctx, Dd, Qd, k)
    kth = gt_d[:, k - 1].clone()

    def recall(ids):
        # squared chord of unit rows (cosine and inner product alike)
        dq = (2.0 - 2.0 * (Qd[:, None, :] * Dd[ids.long().clamp(min=0)]).sum(-1)).clamp(min=0)
        ok = (dq <= kth[:, None] * (1 + 1e-5) + 1e-6) & (ids >= 0)
        return float(ok.sum(1).clamp(max=k).float().mean() / k)

    def curve(idx, beams, prec="fp32"):
        out = []
        for beam in beams:
            idx.search(Qd, k, beam, precision=prec)
            e0, e1 = events()
            e0.record(stream)
            ids, _ = idx.search(Qd, k, beam, precision=prec)
            e1.record(stream)
            torch.cuda.synchronize()
            out.append({"beam": beam, "recall_at_10": recall(ids),
                        "qps": nq / (e0.elapsed_time(e1) / 1e3)})
        return out

    def shape(idx):
        info = idx.info()
        sizes = [int(idx.layer(i)[0].numel()) for i in range(info["n_layers"])]
        dg = idx.layer(0)[2]
        return {"layer_sizes": sizes, "mean_out_degree_layer0": float(dg.float().mean())}

    res = {"workload": w["name"], "n": n, "d": w["d"], "metric": w["metric"], "nq": nq,
           "build_params": f"K 64, L 200, R 32, M 16, I 2, alpha {alpha_it:g} / 60, bf16 "
                           "screen, edge replacement", "data": "synthetic"}
    idx, secs, clk = timed_build(base, 1 if n <= 1_000_000 else 0, Clocks(0))
    res.update({"build_s": secs, "points_per_s": n / secs, "clocks": clk,
                "phase_s": idx.phase_seconds(), **shape(idx),
                "queries": curve(idx, w["beams"]),
                "queries_fp8_screen": curve(idx, w["beams"], "fp8")})
    if c == 4:
        idx.close()
        wider = []
        for af in (70.0, 80.0):
            ix, s2, _ = timed_build(dict(base, alpha_final_deg=af), 0)
            wider.append({"alpha_final": af, "build_s": s2, **shape(ix),
                          "queries": curve(ix, (64, 256))})
            ix.close()
        res["wider_final_alpha"] = wider
    else:
        ins = max(100, n // 100)
        idx.reserve(n + 8 * ins)
        X = synthetic.inserts(c, 8 * ins)
        res["serving"] = serving_measure(pg, idx, Q, X, ins, k, 64, 16)
        idx.close()
    res["autotune"] = pg.autotune_report().splitlines()
    print(json.dumps(res), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.sweep:
        run_sweep(args)
    elif args.extra:
        run_extra(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

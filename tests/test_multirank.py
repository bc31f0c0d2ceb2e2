"""The N > 1 path of bench.py on CPU: two gloo ranks run as replicas; the job
time is the slowest rank's and the rate counts every rank's points."""
from __future__ import annotations

import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [120.0, 250.0][rank]
    ms, rate = bench.job_rate(ms_local, 1000, world)
    dist.barrier()
    q.put((rank, ms, rate))
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in out:
        assert ms == 250.0
        assert rate == pytest.approx(2 * 1000 / 0.25)


def test_single_rank_rate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(500.0, 1000, 1) == (500.0, 2000.0)

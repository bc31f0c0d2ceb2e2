"""The launch-configuration autotuner of the persistent pruning and search
kernels: with tuning on, builds and searches give exactly the results of
untuned runs (the kernels fetch rows from a counter, so any grid gives the
same lists), and the table records the timed candidates."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    import paper_2410_01231_gb300 as pg
    return pg


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_tuned_build_and_search_equal_untuned(pg, precision):
    D, Q, _ = synthetic.workload(1, n=12000, nq=5000)
    Dd, Qd = torch.from_numpy(D).cuda(), torch.from_numpy(Q).cuda()
    prm = dict(K=20, L=64, R=24, M=16, iters=2, precision=precision)
    out = []
    for tune in (False, True):
        ctx = pg.Context()
        ctx.set_autotune(tune)
        idx = pg.Index.build_rng(ctx, Dd, **prm)
        _, nb, dg = idx.layer(0)
        ids, ds = idx.search(Qd, 10, 48)
        out.append((nb.clone(), dg.clone(), ids.clone(), ds.clone()))
        idx.close()
        ctx.close()
    for a, b in zip(out[0], out[1]):
        assert torch.equal(a, b)
    rep = pg.autotune_report()
    assert "k_prune" in rep and "k_search" in rep
    for line in rep.strip().splitlines():
        assert "->" in line and "ms)" in line

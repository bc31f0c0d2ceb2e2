"""Run-twice determinism on the device path: the same input built twice, on
two contexts, gives identical graphs byte for byte (layers, degrees, entry
points) in both precision forms, also on real-valued rows where the
screened kNN, the FP32 decisions and their FP64 rechecks all take part."""
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


def _graph(idx):
    out = [idx.info()]
    for i in range(idx.info()["n_layers"]):
        out.append(tuple(t.cpu().numpy().tobytes() for t in idx.layer(i)))
    return out


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_rng_build_is_deterministic_on_real_rows(pg, precision):
    D, _ = synthetic.mixture_float(8000, 64, 16, 31)
    Dd = torch.from_numpy(D).cuda()
    g = [_graph(pg.Index.build_rng(pg.Context(), Dd, K=24, L=64, R=24, iters=2,
                                   precision=precision)) for _ in range(2)]
    assert g[0] == g[1]


def test_nswg_build_is_deterministic_on_unit_rows(pg):
    D = synthetic.unit_gaussian(6000, 96, 32)
    Dd = torch.from_numpy(D).cuda()
    g = [_graph(pg.Index.build_nswg(pg.Context(), Dd, metric="cosine", K=24, L=48, R=24,
                                    M=16, iters=1, precision="bf16")) for _ in range(2)]
    assert g[0] == g[1]

"""The allocation-free pruning entry point (pg_prune_noalloc).

Callers that may not allocate device memory -- under an allocator or
runtime that owns every device allocation, or with a footprint fixed after
start-up -- prune through pg_prune_noalloc, which keeps its scratch in a
fixed array inside the library.  It must give exactly what pg_prune and the
FP64 oracle give, call after call (the shared scratch keeps the previous
call's contents).
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu


def _candidates(ids: np.ndarray, seed: int):
    """kNN rows plus repeated ids, -1 entries and the row's own id."""
    rng = np.random.default_rng(seed)
    rows = []
    for u in range(ids.shape[0]):
        r = list(ids[u]) + list(rng.choice(ids[u], 3)) + [-1, u]
        rng.shuffle(r)
        rows.append(r)
    off = np.zeros(len(rows) + 1, np.int64)
    off[1:] = np.cumsum([len(r) for r in rows])
    return off, np.concatenate(rows).astype(np.int32)


def test_prune_noalloc_equals_pg_prune_on_two_calls_in_a_row():
    import paper_2410_01231_gb300 as pg

    ctx = pg.Context()
    cases = [
        (synthetic.workload(1, n=3000, nq=1)[0], "l2", 66.0, 24),     # exact integer data
        (synthetic.unit_gaussian(2500, 96, 21), "cosine", 70.0, 16),  # FP64 rechecks
    ]
    for k, (D, metric, alpha, R) in enumerate(cases):
        Dd = torch.from_numpy(D).cuda()
        ids, _ = pg.build_knn(ctx, Dd, 40, metric)
        off, cand = _candidates(ids.cpu().numpy(), 30 + k)
        offd, candd = torch.from_numpy(off).cuda(), torch.from_numpy(cand).cuda()
        ref_nbr, ref_deg = pg.prune(ctx, Dd, offd, candd, R, alpha, metric)
        nbr, deg = pg.prune_noalloc(Dd, offd, candd, R, alpha, metric)
        torch.cuda.synchronize()
        assert torch.equal(deg, ref_deg), k
        assert torch.equal(nbr, ref_nbr), k
        on, odg = oracle.prune(D, off, cand, R, alpha, metric)
        assert (deg.cpu().numpy() == odg).all(), k
        assert (nbr.cpu().numpy() == on).all(), k


def test_prune_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_2410_01231_gb300 as pg

    n = (1 << 20) + 1
    D = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    cand = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(pg.PGError) as e:
        pg.prune_noalloc(D, off, cand, 8, 60.0)
    assert e.value.status == 5

"""Index files on the device path: an index written by pg_index_save and read
back by pg_index_load has the same layers, entry points, parameters and
search results as the original, owns its points (the original and its data
may go), and grows under insertion exactly like the original.  A damaged
file is refused and the context stays usable."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu

PARAM_FIELDS = ("metric", "precision", "K", "L", "R", "M", "alpha_deg", "alpha_final_deg",
                "iters", "connect_final", "route_layers", "seed")


@pytest.fixture(scope="module")
def pg():
    import paper_2410_01231_gb300 as pg
    return pg


@pytest.fixture(scope="module")
def ctx(pg):
    return pg.Context()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


def layers_of(idx):
    out = []
    for i in range(idx.info()["n_layers"]):
        out.append(tuple(host(t) for t in idx.layer(i)))
    return out


def same_index(a, b):
    assert a.info() == b.info()
    (pa, da), (pb, db) = a.params(), b.params()
    assert da == db
    for f in PARAM_FIELDS:
        assert getattr(pa, f) == getattr(pb, f), f
    for i, (la, lb) in enumerate(zip(layers_of(a), layers_of(b))):
        for x, y in zip(la, lb):
            assert x.shape == y.shape and (x == y).all(), i


def test_nswg_round_trip_search_and_insertion(ctx, pg, tmp_path):
    D, Q, _ = synthetic.workload(1, n=3600, nq=50)
    n0 = 2800
    p = dict(K=24, L=48, R=32, M=16, alpha_deg=70.0, iters=1, seed=5)
    Dd = dev(D[:n0])
    a = pg.Index.build_nswg(ctx, Dd, metric="l2", **p)
    path = str(tmp_path / "nswg.pgi")
    a.save(path)
    info = pg.index_file_check(path)
    assert info == dict(n=n0, d=D.shape[1], n_layers=a.info()["n_layers"])
    b = pg.Index.load(ctx, path)
    same_index(a, b)
    ia, da = a.search(dev(Q), 10, 64)
    ib, db = b.search(dev(Q), 10, 64)
    assert (host(ia) == host(ib)).all() and (host(da) == host(db)).all()
    # both grow alike: the loaded index keeps the level draw and the angle
    for idx in (a, b):
        idx.reserve(3600)
        idx.insert(dev(D[n0:3200]), 40, 1)
        idx.insert(dev(D[3200:]), 40, 1)
    same_index(a, b)
    # the loaded index owns its points: the original and its data can go
    a.close()
    a.D = None
    del Dd
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    ib2, db2 = b.search(dev(Q), 10, 64)
    assert (host(ib2) >= 0).all()
    # saving the grown index and loading it again round-trips as well
    path2 = str(tmp_path / "grown.pgi")
    b.save(path2)
    c = pg.Index.load(ctx, path2)
    same_index(b, c)
    ic, dc = c.search(dev(Q), 10, 64)
    assert (host(ic) == host(ib2)).all() and (host(dc) == host(db2)).all()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_rng_round_trip_with_routing_layers(ctx, pg, tmp_path, precision):
    D, Q, _ = synthetic.workload(1, n=4000, nq=64)
    a = pg.Index.build_rng(ctx, dev(D), K=20, L=64, R=24, iters=2, precision=precision)
    path = str(tmp_path / "rng.pgi")
    a.save(path)
    b = pg.Index.load(ctx, path)
    same_index(a, b)
    for flat in (False, True):
        ia, da = a.search(dev(Q), 10, 48, flat=flat)
        ib, db = b.search(dev(Q), 10, 48, flat=flat)
        assert (host(ia) == host(ib)).all() and (host(da) == host(db)).all()


def test_damaged_file_is_refused_and_context_survives(ctx, pg, tmp_path):
    D, Q, _ = synthetic.workload(1, n=1500, nq=16)
    a = pg.Index.build_nswg(ctx, dev(D), metric="l2", K=16, L=32, R=16, M=16, alpha_deg=70.0,
                            iters=1, seed=2)
    path = tmp_path / "ix.pgi"
    a.save(str(path))
    blob = bytearray(path.read_bytes())
    blob[len(blob) // 2] ^= 0x10
    bad = tmp_path / "bad.pgi"
    bad.write_bytes(bytes(blob))
    with pytest.raises(pg.PGError) as e:
        pg.Index.load(ctx, str(bad))
    assert e.value.status == 1
    with pytest.raises(pg.PGError) as e:
        pg.Index.load(ctx, str(tmp_path / "missing.pgi"))
    assert e.value.status == 9
    ids, _ = a.search(dev(Q), 5, 32)
    assert (host(ids) >= 0).all()
    assert not (tmp_path / "ix.pgi.partial").exists()

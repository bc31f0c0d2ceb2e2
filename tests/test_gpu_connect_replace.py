"""Connectivity with edge replacement on the device (a reading of the
connectivity step of Algorithm 2 / Algorithm 5 for graphs whose reached
nodes are all full): pg_connect_replace equals oracle.connect_replace edge
for edge, on tight clusters where the plain step refuses and on random full
graphs (exact integer rows and real rows); builds that used to stop with
PG_ERR_CAPACITY now complete connected."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    import paper_2410_01231_gb300 as pg
    return pg


@pytest.fixture(scope="module")
def ctx(pg):
    return pg.Context()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _reach(nbr, deg, ep):
    seen, stack = {ep}, [ep]
    while stack:
        x = stack.pop()
        for y in nbr[x, :deg[x]]:
            if int(y) not in seen:
                seen.add(int(y))
                stack.append(int(y))
    return seen


def _tight(seed, clusters=12, per=16, d=64, scale=1.0):
    rs = np.random.default_rng(seed)
    centres = rs.normal(0, 10, (clusters, d))
    D = np.vstack([c + rs.normal(0, 0.05, (per, d)) for c in centres]) * scale
    return D.astype(np.float32)


@pytest.mark.parametrize("kind", ["real", "int"])
def test_replacement_links_full_tight_clusters_like_the_oracle(ctx, pg, kind):
    # integer rows: exact FP32 distances (partial sums below 2^24), one pass
    D = _tight(41) if kind == "real" else np.rint(_tight(41, scale=6.0)).astype(np.float32)
    n, K, R = D.shape[0], 8, 4
    ids, _ = oracle.knn(D, K)
    nbr, deg = oracle.prune(D, np.arange(n + 1, dtype=np.int64) * K, ids.ravel(), R, 66.0)
    ep = oracle.medoid(D)
    if oracle.connect(D, nbr, deg, ep)[2] >= 0:
        pytest.skip("the plain step does not refuse on this draw")
    with pytest.raises(pg.PGError) as e:
        pg.connect(ctx, dev(D), dev(nbr), dev(deg), ep)
    assert e.value.status == 5
    gn, gd = dev(nbr), dev(deg)
    added, rep = pg.connect_replace(ctx, dev(D), gn, gd, ep)
    on, od, oadded, orep = oracle.connect_replace(D, nbr, deg, ep)
    assert (added, rep) == (oadded, orep) and rep > 0
    assert (gd.cpu().numpy() == od).all() and (gn.cpu().numpy() == on).all()


@pytest.mark.parametrize("seed", range(6))
def test_replacement_equals_the_oracle_on_random_full_graphs(ctx, pg, seed):
    rs = np.random.default_rng(900 + seed)
    n, R = int(rs.integers(30, 400)), int(rs.integers(1, 5))
    d = 16
    D = rs.integers(0, 6, size=(n, d)).astype(np.float32)
    if seed % 2:
        D = D * np.float32(0.37) + rs.normal(0, 0.01, (n, d)).astype(np.float32)
    nbr = np.full((n, R), -1, np.int32)
    deg = np.full(n, R, np.int32)
    deg[rs.random(n) < 0.1] = 0
    for u in range(n):
        nbr[u, :deg[u]] = rs.choice(n, size=deg[u], replace=True)
    ep = int(rs.integers(0, n))
    on, od, oadded, orep = oracle.connect_replace(D, nbr, deg, ep)
    gn, gd = dev(nbr), dev(deg)
    if oadded < 0:
        with pytest.raises(pg.PGError):
            pg.connect_replace(ctx, dev(D), gn, gd, ep)
        return
    added, rep = pg.connect_replace(ctx, dev(D), gn, gd, ep)
    assert (added, rep) == (oadded, orep)
    assert (gd.cpu().numpy() == od).all() and (gn.cpu().numpy() == on).all()
    assert _reach(gn.cpu().numpy(), gd.cpu().numpy(), ep) == set(range(n))


def test_replacement_equals_plain_step_when_plain_succeeds(ctx, pg):
    D, _, _ = synthetic.workload(1, n=3000, nq=1)
    ids, _ = oracle.knn(D, 8)
    nbr, deg = oracle.prune(D, np.arange(3001, dtype=np.int64) * 8, ids.ravel(), 16, 60.0)
    ep = oracle.medoid(D)
    a_n, a_d = dev(nbr), dev(deg)
    b_n, b_d = dev(nbr), dev(deg)
    plain = pg.connect(ctx, dev(D), a_n, a_d, ep)
    added, rep = pg.connect_replace(ctx, dev(D), b_n, b_d, ep)
    assert (added, rep) == (plain, 0)
    assert torch.equal(a_n, b_n) and torch.equal(a_d, b_d)


def test_build_on_full_tight_clusters_completes_connected(ctx, pg):
    D = _tight(43, clusters=24, per=24)
    prm = dict(K=12, L=24, R=4, M=16, alpha_deg=66.0, alpha_final_deg=66.0, iters=1,
               route_layers=0)
    with pytest.raises(pg.PGError) as e:
        pg.Index.build_rng(ctx, dev(D), connect_replace=0, **prm)
    assert e.value.status == 5
    idx = pg.Index.build_rng(ctx, dev(D), **prm)
    _, nb, dg = idx.layer(0)
    nb, dg = nb.cpu().numpy(), dg.cpu().numpy()
    assert (dg <= 4).all()
    assert _reach(nb, dg, idx.info()["ep_base"]) == set(range(D.shape[0]))
    idx.close()

"""The input recipe (CPU): shapes, value sets, norms, determinism and the
cluster structure of the seeded generators that stand in for the paper's
datasets, at reduced sizes."""
import numpy as np
import pytest

import synthetic


def test_byte_mixture_values_and_clusters():
    D, c = synthetic.mixture_int(5000, 128, 32, 1)
    assert D.dtype == np.float32 and D.shape == (5000, 128) and c.shape == (32, 128)
    assert (D == np.rint(D)).all() and D.min() >= 0 and D.max() <= 255
    # every row lies near one of the 32 centres (sigma 20 per coordinate)
    d2 = ((D[:, None, :].astype(np.float64) - c[None]) ** 2).sum(-1).min(1)
    assert np.sqrt(d2 / 128).max() < 25


def test_real_mixture_and_unit_rows():
    D, c = synthetic.mixture_float(3000, 96, 16, 2)
    assert D.dtype == np.float32 and (D != np.rint(D)).any()
    assert abs(float((D - c[np.argmin(((D[:, None] - c[None]) ** 2).sum(-1), 1)]).std()) - 0.1) < 0.01
    U = synthetic.unit_gaussian(2000, 96, 3)
    assert np.allclose(np.linalg.norm(U.astype(np.float64), axis=1), 1, atol=1e-6)
    S, sc = synthetic.sphere_mixture(2000, 384, 64, 4)
    assert np.allclose(np.linalg.norm(S.astype(np.float64), axis=1), 1, atol=1e-6)
    assert np.allclose(np.linalg.norm(sc, axis=1), 1)


@pytest.mark.parametrize("c", [1, 2, 3, 4, 5])
def test_workloads_are_deterministic_and_shaped(c):
    D1, Q1, w = synthetic.workload(c, n=700, nq=30)
    D2, Q2, _ = synthetic.workload(c, n=700, nq=30)
    assert (D1 == D2).all() and (Q1 == Q2).all()
    assert D1.shape == (700, w["d"]) and Q1.shape == (30, w["d"])
    assert D1.dtype == np.float32 and Q1.dtype == np.float32
    full = synthetic.WORKLOADS[c]
    assert w["d"] == full["d"] and w["metric"] == full["metric"]
    if full["kind"] in ("unit", "sphere"):
        assert np.allclose(np.linalg.norm(D1.astype(np.float64), axis=1), 1, atol=1e-6)


def test_queries_share_the_points_centres():
    D, Q, _ = synthetic.workload(1, n=4000, nq=200)
    _, c = synthetic.mixture_int(1, 128, 32, 1234 + 1)
    dq = ((Q[:, None, :].astype(np.float64) - c[None]) ** 2).sum(-1).min(1)
    assert np.sqrt(dq / 128).max() < 25
    X = synthetic.inserts(1, 100)
    dx = ((X[:, None, :].astype(np.float64) - c[None]) ** 2).sum(-1).min(1)
    assert X.shape == (100, 128) and np.sqrt(dx / 128).max() < 25

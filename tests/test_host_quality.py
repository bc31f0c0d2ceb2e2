"""Host logic of the quality examination (Section 5.2), on CPU: the
library's Theorem 3 sample size equals the oracle's, and the builds' sample
is a set of distinct, ascending ids of [0, n) that covers the range evenly."""
from __future__ import annotations

import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def pg():
    import paper_2410_01231_gb300 as pg
    return pg


@pytest.mark.parametrize("n", [2, 10, 1000, 1_000_000, 2_000_000_000])
@pytest.mark.parametrize("eps", [0.05, 0.3, 0.6, 1.0])
@pytest.mark.parametrize("l", [1.0, 2.0])
def test_sample_size_equals_the_oracle(pg, n, eps, l):
    assert pg.quality_sample_size(n, eps, l) == oracle.quality_sample_size(n, eps, l)


def test_sample_size_refuses_bad_arguments(pg):
    assert pg.quality_sample_size(1, 0.6) == -1
    assert pg.quality_sample_size(100, 0.0) == -1
    assert pg.quality_sample_size(100, 0.6, 0.0) == -1


@pytest.mark.parametrize("n,ns,seed", [(1, 1, 0), (10, 10, 3), (1000, 353, 0), (50_000, 353, 7)])
def test_sample_is_distinct_sorted_and_in_range(pg, n, ns, seed):
    s = pg.quality_sample(n, ns, seed)
    assert s.shape == (ns,) and s.dtype == np.int32
    assert (np.diff(s) > 0).all() and s.min() >= 0 and s.max() < n
    assert (pg.quality_sample(n, ns, seed) == s).all()


def test_sample_covers_the_range_evenly(pg):
    n, ns = 1_000_000, 20_000
    s = pg.quality_sample(n, ns, 11)
    hist, _ = np.histogram(s, bins=10, range=(0, n))
    assert (np.abs(hist - ns / 10) < 5 * np.sqrt(ns / 10)).all(), hist
    assert not np.array_equal(s, pg.quality_sample(n, ns, 12))

"""The library's level draw for NSWG layers and insertion (pg_levels, host
code of libpg, no device) equals the oracle's restatement of Algorithm 7's
draw (whose SplitMix64 is pinned by published outputs) for several seeds and
level bases."""
import numpy as np
import pytest

import oracle
import paper_2410_01231_gb300 as pg


@pytest.mark.parametrize("seed", [0, 1, 977, 2**40 + 3, 2**64 - 1])
@pytest.mark.parametrize("M", [2, 16, 64])
def test_library_levels_equal_the_oracle(seed, M):
    n = 50_000
    assert (pg.levels(n, seed, M) == oracle.levels(n, seed, M)).all()


def test_level_histogram_follows_the_geometric_law():
    lev = pg.levels(400_000, 7, 16)
    frac = np.bincount(lev) / lev.size
    # P(l >= i) = 16^-i
    assert frac[0] == pytest.approx(1 - 1 / 16, abs=2e-3)
    assert (frac[1:3].sum()) == pytest.approx(1 / 16 - 1 / 16 ** 3, rel=3e-2)


def test_levels_argument_checks():
    assert pg.levels(0, 1, 16).shape == (0,)
    with pytest.raises(pg.PGError):
        pg.levels(10, 1, 1)

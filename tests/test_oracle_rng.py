"""Pins of the oracle's random numbers (§2.2: pseudo-random normals).

Philox4x32-10 is pinned to the generator's published known-answer vectors;
the Box-Muller normals are pinned statistically (moments, independence and a
Kolmogorov-Smirnov test against the exact N(0,1) law), which a wrong constant
(2 pi vs pi, -2 ln vs -ln), a swapped uniform or a reused word would fail.
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], tuple(w[6:10])))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(orc, ctr, key, expect):
    assert orc.philox4x32_10(ctr, key) == expect


def _many_normals(orc, count_pairs=40000, seed=12345):
    z = np.empty((count_pairs, 4))
    for q in range(count_pairs):
        z[q] = orc.normals(seed, q % 97, q // 97, q % 5)
    return z


def test_normals_moments_and_independence(orc):
    z = _many_normals(orc)
    flat = z.ravel()
    m = flat.size
    assert abs(flat.mean()) < 4.0 / math.sqrt(m)
    assert abs(flat.var() - 1.0) < 4.0 * math.sqrt(2.0 / m)
    kurt = np.mean(flat ** 4)
    assert abs(kurt - 3.0) < 4.0 * math.sqrt(96.0 / m)
    # the two components of a pair and the two pairs of a block are uncorrelated
    for a, b in ((0, 1), (2, 3), (0, 2), (1, 3)):
        r = np.corrcoef(z[:, a], z[:, b])[0, 1]
        assert abs(r) < 4.0 / math.sqrt(z.shape[0])
    # squares of the two components of a pair are uncorrelated too (a pair
    # from R cos / R sin with a wrong radius law fails this)
    r2 = np.corrcoef(z[:, 0] ** 2, z[:, 1] ** 2)[0, 1]
    assert abs(r2) < 4.0 / math.sqrt(z.shape[0])


def test_normals_distribution_ks(orc):
    from scipy import stats
    z = _many_normals(orc, count_pairs=20000, seed=7)
    for c in range(4):
        res = stats.kstest(z[:, c], "norm")
        assert res.pvalue > 1e-4, (c, res)
    # radius of a pair: R^2 = z0^2 + z1^2 is exponential with mean 2
    r2 = z[:, 0] ** 2 + z[:, 1] ** 2
    assert stats.kstest(r2, "expon", args=(0.0, 2.0)).pvalue > 1e-4


def test_normals_depend_on_every_counter_word(orc):
    base = orc.normals(1, 2, 3, 4)
    for args in ((2, 2, 3, 4), (1, 3, 3, 4), (1, 2, 4, 4), (1, 2, 3, 5), (1 << 32 | 1, 2, 3, 4)):
        assert not np.allclose(orc.normals(*args), base)

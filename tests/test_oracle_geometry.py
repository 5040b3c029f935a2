"""Pins of the oracle's per-step pieces: density and drift (eq.
WinslowTypeGridGeneratorExpanded), exit test and exit point (§2.2), boundary
lookup, and the interface-node plan (§2.1, Fig. 1)."""
import math

import numpy as np
import pytest

import workloads as W

FAMILIES = [
    (W.FAMILY_BUMPS, W.bumps((5.0, 0.5, 0.5, 50.0, 50.0))),
    (W.FAMILY_BUMPS, W.bumps((8.0, 0.3, 0.6, 30.0, 10.0), (3.0, 0.7, 0.2, 80.0, 80.0))),
    (W.FAMILY_RING, (10.0, 0.5, 0.5, 50.0, 0.25)),
    (W.FAMILY_RIDGE, (20.0, 200.0, 0.3, 0.2, 1.0)),
]


@pytest.mark.parametrize("family,params", FAMILIES)
@pytest.mark.parametrize("coef_mode", [W.COEF_W, W.COEF_INV_W])
def test_drift_is_gradient_of_log_coefficient(orc, family, params, coef_mode):
    """b = grad ln c, checked against central differences of ln c."""
    rng = np.random.default_rng(1)
    h = 1e-6
    for s, t in rng.uniform(0.02, 0.98, size=(40, 2)):
        b = orc.drift(family, coef_mode, params, s, t)
        lc = lambda a, c: math.log(float(orc.coef(family, coef_mode, params, a, c)))
        gs = (lc(s + h, t) - lc(s - h, t)) / (2 * h)
        gt = (lc(s, t + h) - lc(s, t - h)) / (2 * h)
        scale = 1.0 + abs(gs) + abs(gt)
        assert abs(b[0] - gs) < 1e-5 * scale, (s, t, b, gs)
        assert abs(b[1] - gt) < 1e-5 * scale, (s, t, b, gt)


def test_density_values_at_features(orc):
    A = 5.0
    p = W.bumps((A, 0.5, 0.5, 50.0, 50.0))
    assert orc.coef(W.FAMILY_BUMPS, W.COEF_W, p, 0.5, 0.5) == pytest.approx(1 + A)
    assert orc.coef(W.FAMILY_BUMPS, W.COEF_INV_W, p, 0.5, 0.5) == pytest.approx(1 / (1 + A))
    # exp(-50 * 0.1^2) at distance 0.1
    assert orc.coef(W.FAMILY_BUMPS, W.COEF_W, p, 0.6, 0.5) == pytest.approx(
        1 + A * math.exp(-0.5))
    ring = (10.0, 0.5, 0.5, 50.0, 0.25)
    assert orc.coef(W.FAMILY_RING, W.COEF_W, ring, 0.75, 0.5) == pytest.approx(11.0)
    assert orc.coef(W.FAMILY_RING, W.COEF_W, ring, 0.5, 0.5) == pytest.approx(
        1 + 10 / math.cosh(12.5) ** 2)
    ridge = (20.0, 200.0, 0.3, 0.2, 1.0)
    assert orc.coef(W.FAMILY_RIDGE, W.COEF_W, ridge, 0.25, 0.5) == pytest.approx(21.0)
    assert orc.coef(W.FAMILY_RIDGE, W.COEF_W, ridge, 0.0, 0.3) == pytest.approx(21.0)
    # no bumps: c = 1 and no drift
    assert orc.coef(W.FAMILY_BUMPS, W.COEF_W, (0.0,), 0.3, 0.7) == 1.0
    assert np.all(orc.drift(W.FAMILY_BUMPS, W.COEF_W, (0.0,), 0.3, 0.7) == 0.0)
    # the drift points up the density for c = w and down for c = 1/w
    b = orc.drift(W.FAMILY_BUMPS, W.COEF_W, p, 0.4, 0.5)
    assert b[0] > 0 and abs(b[1]) < 1e-12
    b = orc.drift(W.FAMILY_BUMPS, W.COEF_INV_W, p, 0.4, 0.5)
    assert b[0] < 0


def test_exit_point_cases(orc):
    # inside: no exit
    assert orc.exit_point(0.5, 0.5, 0.6, 0.4)[0] == -1
    # crosses s = 1 at t = 0.55
    e, p = orc.exit_point(0.9, 0.5, 1.1, 0.6)
    assert e == 3 and p[0] == 1.0 and p[1] == pytest.approx(0.55)
    # crosses s = 0
    e, p = orc.exit_point(0.1, 0.5, -0.1, 0.3)
    assert e == 2 and p[0] == 0.0 and p[1] == pytest.approx(0.4)
    # crosses t = 0 and t = 1
    e, p = orc.exit_point(0.5, 0.05, 0.7, -0.05)
    assert e == 0 and p[1] == 0.0 and p[0] == pytest.approx(0.6)
    e, p = orc.exit_point(0.2, 0.9, 0.4, 1.3)
    assert e == 1 and p[1] == 1.0 and p[0] == pytest.approx(0.25)
    # corner region: both sides violated, the earlier crossing wins
    e, p = orc.exit_point(0.9, 0.95, 1.3, 1.05)      # theta_s = .25, theta_t = .5
    assert e == 3 and p[1] == pytest.approx(0.975)
    e, p = orc.exit_point(0.95, 0.9, 1.05, 1.3)      # theta_s = .5, theta_t = .25
    assert e == 1 and p[0] == pytest.approx(0.975)
    # exact tie goes to the s-side
    e, p = orc.exit_point(0.9, 0.9, 1.1, 1.1)
    assert e == 3 and p == pytest.approx([1.0, 1.0])
    # landing exactly on a side counts as an exit (closed sides)
    e, p = orc.exit_point(0.9, 0.5, 1.0, 0.5)
    assert e == 3 and p[1] == 0.5
    e, p = orc.exit_point(0.5, 0.1, 0.5, 0.0)
    assert e == 0


def test_lookup_is_linear_interpolation(orc):
    n = 9
    T = np.arange(n) / (n - 1.0)
    for tau in (0.0, 0.125, 0.3, 0.5, 0.77, 1.0):
        assert orc.lookup(T, tau) == pytest.approx(tau, abs=1e-15)
    T2 = np.array([0.0, 1.0, 4.0, 9.0, 16.0])
    assert orc.lookup(T2, 0.25) == 1.0
    assert orc.lookup(T2, 0.375) == pytest.approx(2.5)
    assert orc.lookup(T2, 1.0) == 16.0
    assert orc.lookup(np.full(5, 0.7), 0.61) == 0.7


@pytest.mark.parametrize("n,sx,sy,expect", [(33, 2, 2, 61), (257, 4, 4, 1521),
                                            (1025, 8, 8, 14273), (17, 2, 3, 43),
                                            (9, 1, 1, 0), (5, 4, 4, 9)])
def test_interface_node_counts(orc, n, sx, sy, expect):
    nodes = orc.interface_nodes(n, sx, sy)
    assert len(nodes) == expect
    assert len({(int(i), int(j)) for i, j in nodes}) == expect
    # ordered by row, then column
    key = [(int(j), int(i)) for i, j in nodes]
    assert key == sorted(key)


def test_interface_indices_rule(orc):
    assert orc.interface_indices(33, 2) == [16]
    assert orc.interface_indices(257, 4) == [64, 128, 192]
    # n-1 = 64 split 3 ways: 21.33 -> 21, 42.67 -> 43
    assert orc.interface_indices(65, 3) == [21, 43]
    # 7 ways of 128: 18.29, 36.57, 54.86, 73.14, 91.43, 109.71
    assert orc.interface_indices(129, 7) == [18, 37, 55, 73, 91, 110]
    # a half rounds up: 2 ways of 9 intervals -> 4.5 -> 5
    assert orc.interface_indices(10, 2) == [5]


@pytest.mark.parametrize("n,sx,sy", [(33, 2, 2), (65, 3, 5), (20, 4, 2)])
def test_subdomains_partition_the_interior(orc, n, sx, sy):
    seen = np.zeros((n, n), dtype=int)
    for (i0, i1, j0, j1) in orc.subdomains(n, sx, sy):
        seen[j0 + 1:j1, i0 + 1:i1] += 1
    nodes = orc.interface_nodes(n, sx, sy)
    seen[nodes[:, 1], nodes[:, 0]] += 1
    assert np.all(seen[1:-1, 1:-1] == 1)
    assert np.all(seen[0, :] == 0) and np.all(seen[:, 0] == 0)

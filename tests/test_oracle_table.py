"""Pins of the oracle's tabulated density (w = exp(L), L the bilinear
interpolant of a table of ln w; drift = sgn grad L): exactness for linear
tables, interpolation of the nodes, convergence to an analytic density as the
table is refined, and the 1D closed form, which ties the drift to the
coefficient used by the finite-difference operator."""
import math

import numpy as np
import pytest

import workloads as W

T = W.FAMILY_TABLE


def _nodes(tn):
    x = np.arange(tn) / (tn - 1.0)
    return np.meshgrid(x, x, indexing="xy")


@pytest.mark.parametrize("coef_mode", [W.COEF_W, W.COEF_INV_W])
def test_bilinear_table_gives_the_exact_drift(orc, coef_mode):
    """L = a s + b t + k s t is reproduced exactly by bilinear interpolation:
    the drift is (a + k t, b + k s) (times the coefficient sign) everywhere,
    cell edges included, and c = exp(+-L)."""
    tn, a, b, k = 9, 1.7, -0.6, 2.3
    S, Tt = _nodes(tn)
    p = W.table_params(a * S + b * Tt + k * S * Tt)
    sgn = 1.0 if coef_mode == W.COEF_W else -1.0
    rng = np.random.default_rng(1)
    pts = list(rng.random((50, 2))) + [(0.5, 0.5), (0.25, 0.125), (1.0, 1.0), (0.0, 0.0)]
    for s, t in pts:
        d = orc.drift(T, coef_mode, p, float(s), float(t))
        assert np.allclose(d, [sgn * (a + k * t), sgn * (b + k * s)], rtol=0, atol=1e-12)
        c = orc.coef(T, coef_mode, p, s, t)
        assert c == pytest.approx(math.exp(sgn * (a * s + b * t + k * s * t)), rel=1e-13)


def test_table_interpolates_its_nodes_and_is_continuous(orc):
    tn = 7
    L = W.smooth_field(tn, seed=3, amplitude=1.5)
    p = W.table_params(L)
    S, Tt = _nodes(tn)
    w = orc.coef(T, W.COEF_W, p, S, Tt)
    assert np.allclose(np.log(w), L, rtol=0, atol=1e-14)
    # continuous across a cell edge, the gradient jumps only in the tangential
    # interpolation weight
    e = 1e-9
    x0 = 2.0 / (tn - 1)
    for t in (0.1, 0.37, 0.9):
        left = orc.coef(T, W.COEF_W, p, x0 - e, t)
        right = orc.coef(T, W.COEF_W, p, x0 + e, t)
        assert left == pytest.approx(right, rel=1e-7)


def test_tabulated_bump_converges_to_the_analytic_bump(orc):
    """ln w of the analytic bump family sampled on tn x tn nodes: the
    single-domain finite-difference mesh of the table converges to the
    analytic one at second order in the table spacing."""
    n = 33
    fam, p = W.FAMILY_BUMPS, W.bumps((5.0, 0.5, 0.5, 30.0, 30.0))
    E = orc.bmap_tables(n, W.BMAP_IDENTITY)
    G = orc.global_solve(n, E, fam, W.COEF_W, p)
    err = []
    for tn in (13, 25, 49):           # nodes never on the operator's edge midpoints
        S, Tt = _nodes(tn)
        lw = np.log(orc.coef(fam, W.COEF_W, p, S, Tt))
        H = orc.global_solve(n, E, T, W.COEF_W, W.table_params(lw))
        err.append(np.max(np.abs(H - G)))
    assert err[-1] < 2e-3, err
    assert 2.5 < err[0] / err[1] < 6 and 2.5 < err[1] / err[2] < 6, err


def test_table_in_s_matches_the_one_dimensional_closed_form(orc):
    """L = L(s): the Monte Carlo estimate (whose drift is grad L) agrees within
    3 sigma + bias with phi(s) = int c^-1 / int c^-1 for c = exp(L), the
    coefficient of the finite-difference operator and of the quadrature."""
    tn, n = 33, 33
    S, Tt = _nodes(tn)
    L = 1.2 * np.sin(2.5 * S) + 0.8 * S * S
    p = W.table_params(L)
    phi = lambda x: orc.closed_form_1d(T, W.COEF_W, p, x, axis=0)
    x = np.arange(n) / (n - 1.0)
    E = np.zeros((2, 4, n))
    E[0, 0] = phi(x); E[0, 1] = E[0, 0]; E[0, 2] = 0.0; E[0, 3] = 1.0
    E[1, 2] = x; E[1, 3] = x; E[1, 0] = 0.0; E[1, 1] = 1.0
    nodes = orc.interface_nodes(n, 2, 2)[::3]
    r = orc.mc_nodes(n, nodes, E, T, W.COEF_W, p, seed=6, paths=4000, dt=1e-4,
                     max_steps=10 ** 5, exit_test=1)
    mean, se = orc.mc_estimate(nodes, n, r["S_all"], r["Q_all"], r["paths"])
    exact = np.c_[phi(nodes[:, 0] / (n - 1.0)), nodes[:, 1] / (n - 1.0)]
    z = np.abs(mean - exact) / se
    assert (z > 3.5).sum() <= 1, z.max()
    # the drift's sign matters: the reversed drift is far off
    r2 = orc.mc_nodes(n, nodes, E, T, W.COEF_INV_W, p, seed=6, paths=4000, dt=1e-4,
                      max_steps=10 ** 5, exit_test=1)
    m2, _ = orc.mc_estimate(nodes, n, r2["S_all"], r2["Q_all"], r2["paths"])
    assert np.max(np.abs(m2 - exact)[:, 0] / se[:, 0]) > 8.0


def test_constant_table_is_the_identity(orc):
    n = 17
    p = W.table_params(np.full((5, 5), 0.7))
    E = orc.bmap_tables(n, W.BMAP_IDENTITY)
    G = orc.global_solve(n, E, T, W.COEF_W, p)
    x = np.arange(n) / (n - 1.0)
    assert np.max(np.abs(G[:, :, 0] - x[None, :])) < 1e-13
    assert orc.drift(T, W.COEF_W, p, 0.3, 0.6) == pytest.approx([0.0, 0.0], abs=0)

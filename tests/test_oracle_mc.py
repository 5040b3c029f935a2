"""Pins of the oracle's Monte Carlo estimate (§2.1-2.2) against what the
mathematics fixes: harmonic (identity) solutions for c = 1, the closed-form 1D
solution u = int c^-1 / int c^-1 (§3.2's 1D forms), the mean exit time of
sqrt(2) W from the square (noise scale), symmetry, and agreement with the
single-domain finite-difference mesh (§3.2-3.5).  Each closed-form pin also
checks that the wrong readings of the SDE (drift sign, noise scale 1 instead
of sqrt 2) would have been caught."""
import math

import numpy as np
import pytest

import workloads as W


def _est(orc, n, nodes, r, nt=False):
    S = r["S_nt"] if nt else r["S_all"]
    Q = r["Q_nt"] if nt else r["Q_all"]
    N = r["paths"] - (r["ties"] if nt else 0)
    return orc.mc_estimate(nodes, n, S, Q, N)


def test_constant_coefficient_identity_is_unbiased(orc):
    """c = 1, identity map: E[F] = X0 (linear functions are harmonic)."""
    n = 9
    E = orc.bmap_tables(n, W.BMAP_IDENTITY)
    nodes = orc.interface_nodes(n, 2, 2)
    r = orc.mc_nodes(n, nodes, E, W.FAMILY_BUMPS, W.COEF_W, (0.0,), seed=21, paths=2000,
                     dt=1e-5, max_steps=400000, tie_delta=1e-11)
    mean, se = _est(orc, n, nodes, r)
    z = np.abs(mean - nodes / (n - 1.0)) / se
    assert np.sum(z > 3.0) <= max(1, math.ceil(0.01 * z.size)), z
    assert r["non_exits"].sum() == 0


def _table_from(orc, n, comp_fn_s, comp_fn_t):
    """Boundary tables of the exact solution u = (U1(s), U2(t))."""
    x = np.arange(n) / (n - 1.0)
    E = np.zeros((2, 4, n))
    E[0, 0] = comp_fn_s(x); E[0, 1] = comp_fn_s(x)
    E[0, 2] = comp_fn_s(np.array([0.0]))[0]; E[0, 3] = comp_fn_s(np.array([1.0]))[0]
    E[1, 2] = comp_fn_t(x); E[1, 3] = comp_fn_t(x)
    E[1, 0] = comp_fn_t(np.array([0.0]))[0]; E[1, 1] = comp_fn_t(np.array([1.0]))[0]
    return E


def _alternatives(orc, fam, coef_mode, p, x, axis):
    """Wrong readings: opposite drift sign (int c / int c) and unit noise with
    drift grad ln c (generator Lap/2 + grad ln c . grad: int c^-2 / int c^-2)."""
    from scipy.integrate import quad

    def cf(y):
        s, t = (y, 0.5) if axis == 0 else (0.5, y)
        return float(orc.coef(fam, coef_mode, p, s, t))

    out = []
    for g in (lambda y: cf(y), lambda y: cf(y) ** -2):
        tot = quad(g, 0, 1, limit=200)[0]
        out.append(np.array([quad(g, 0, v, limit=200)[0] / tot for v in x]))
    return out


@pytest.mark.parametrize("case", ["s_bump_w", "t_ridge_invw"])
def test_one_dimensional_closed_form(orc, case):
    """c depends on one coordinate: u = (phi(s), t) or (s, phi(t)) with
    phi = int_0^x c^-1 / int_0^1 c^-1."""
    n = 65
    if case == "s_bump_w":
        fam, cm, p, axis = W.FAMILY_BUMPS, W.COEF_W, W.bumps((6.0, 0.35, 0.0, 40.0, 0.0)), 0
    else:
        fam, cm, p, axis = W.FAMILY_RIDGE, W.COEF_INV_W, (6.0, 40.0, 0.62, 0.0, 1.0), 1
    phi = lambda x: orc.closed_form_1d(fam, cm, p, x, axis=axis)
    ident = lambda x: np.asarray(x, dtype=float)
    E = _table_from(orc, n, phi, ident) if axis == 0 else _table_from(orc, n, ident, phi)
    nodes = orc.interface_nodes(n, 2, 2)
    nodes = nodes[::6]
    r = orc.mc_nodes(n, nodes, E, fam, cm, p, seed=5, paths=4000, dt=2e-5,
                     max_steps=200000, tie_delta=1e-11)
    mean, se = _est(orc, n, nodes, r)
    x = nodes / (n - 1.0)
    exact = np.empty_like(mean)
    exact[:, axis] = phi(x[:, axis])
    exact[:, 1 - axis] = x[:, 1 - axis]
    # MC error + O(sqrt(dt)) exit bias + O(h^2) boundary interpolation
    tol = 3.0 * se + 2.5e-3
    bad = np.abs(mean - exact) > tol
    assert bad.sum() <= 1, np.c_[x, mean, exact, se][bad.any(axis=1)]
    # the pin separates the readings of the SDE
    for alt in _alternatives(orc, fam, cm, p, x[:, axis], axis):
        assert np.max(np.abs(alt - exact[:, axis]) / se[:, axis]) > 8.0


@pytest.mark.parametrize("s0,t0", [(0.5, 0.5), (0.5, 0.25), (0.25, 0.5)])
def test_mean_exit_time_fixes_the_noise_scale(orc, s0, t0):
    """c = 1: E[tau] solves Lap v = -1 (generator Lap of sqrt(2) W).  Plain
    Euler-Maruyama with an end-of-step exit test exits an effectively larger
    square; the shift 0.5826 sqrt(2 dt) per side (Siegmund's correction for a
    discretely monitored Gaussian walk) accounts for that to first order."""
    n = 5
    i, j = int(round(s0 * (n - 1))), int(round(t0 * (n - 1)))
    E = orc.bmap_tables(n, W.BMAP_IDENTITY)
    dt = 1e-5
    r = orc.mc_nodes(n, [(i, j)], E, W.FAMILY_BUMPS, W.COEF_W, (0.0,), seed=9,
                     paths=4000, dt=dt, max_steps=10 ** 6)
    # sample std of tau from one path's worth of replays is not stored; bound it
    # by the path-level estimate below
    taus = np.array([orc.path(n, s0, t0, 0, q, E, W.FAMILY_BUMPS, W.COEF_W, (0.0,), 9, dt,
                              10 ** 6)["steps"] for q in range(4000)], dtype=float) * dt
    assert taus.sum() == pytest.approx(float(r["steps"][0]) * dt, rel=1e-12)
    mean = taus.mean()
    se = taus.std(ddof=1) / math.sqrt(taus.size)
    d = 0.5826 * math.sqrt(2 * dt)
    L = 1.0 + 2 * d
    corrected = L * L * orc.torsion_exit_time((s0 + d) / L, (t0 + d) / L)
    assert abs(mean - corrected) < 4.0 * se, (mean, corrected, se)
    # unit noise would double the exit time
    assert abs(2.0 * corrected - mean) > 20.0 * se


def test_symmetric_density_gives_symmetric_estimates(orc):
    """c symmetric about s = 1/2, identity map: E u1(s,t) + E u1(1-s,t) = 1."""
    n = 17
    p = W.bumps((9.0, 0.5, 0.3, 30.0, 30.0))
    E = orc.bmap_tables(n, W.BMAP_IDENTITY)
    left = np.array([(i, 8) for i in (2, 4, 6)])
    right = np.array([(n - 1 - i, 8) for i in (2, 4, 6)])
    both = np.vstack([left, right])
    r = orc.mc_nodes(n, both, E, W.FAMILY_BUMPS, W.COEF_W, p, seed=4, paths=3000,
                     dt=2e-5, max_steps=200000)
    mean, se = _est(orc, n, both, r)
    s = mean[:3, 0] + mean[3:, 0]
    sse = np.sqrt(se[:3, 0] ** 2 + se[3:, 0] ** 2)
    assert np.all(np.abs(s - 1.0) < 3.5 * sse), (s, sse)


def test_estimates_approach_the_finite_difference_mesh(orc):
    """The interface estimates agree with the single-domain solution of the
    generator (§3.2, §3.5: R = 1 for the DD mesh) up to MC error, the EM exit
    bias and the FD discretisation error (FD taken on a 4x finer grid)."""
    n, fine = 33, 129
    spec = W.config1()
    E = orc.bmap_tables(n, W.BMAP_IDENTITY)
    Ef = orc.bmap_tables(fine, W.BMAP_IDENTITY)
    G = orc.global_solve(fine, Ef, spec.family, spec.coef_mode, spec.params)
    nodes = orc.interface_nodes(n, 2, 2)[::4]
    r = orc.mc_nodes(n, nodes, E, spec.family, spec.coef_mode, spec.params, seed=0,
                     paths=4000, dt=2e-5, max_steps=100000)
    mean, se = _est(orc, n, nodes, r)
    ref = G[nodes[:, 1] * 4, nodes[:, 0] * 4, :]
    tol = 3.0 * se + 2e-3
    assert np.sum(np.abs(mean - ref) > tol) <= 1, np.c_[nodes, mean, ref, se]


def test_node_sums_are_the_sum_of_single_paths(orc):
    n = 17
    spec = W.small_parity_cases()[1]
    E = orc.bmap_tables(n, W.BMAP_IDENTITY)
    node = (4, 11)
    r = orc.mc_nodes(n, [node], E, spec.family, spec.coef_mode, spec.params, seed=77,
                     paths=60, dt=1e-4, max_steps=20000, tie_delta=1e-3,
                     node_ids=[123], path_begin=1000)
    x0 = np.array(node) / (n - 1.0)
    d = []
    ties = steps = 0
    for q in range(1000, 1060):
        pr = orc.path(n, x0[0], x0[1], 123, q, E, spec.family, spec.coef_mode, spec.params,
                      77, 1e-4, 20000, 1e-3)
        d.append((pr["F"] - x0, pr["tie"]))
        ties += pr["tie"]
        steps += pr["steps"]
    dd = np.array([a for a, _ in d])
    tie = np.array([b for _, b in d])
    assert r["paths"][0] == 60 and r["ties"][0] == ties and r["steps"][0] == steps
    assert ties > 0                      # a wide tie band flags some paths
    assert np.allclose(r["S_all"][0], dd.sum(0), rtol=1e-13, atol=1e-15)
    assert np.allclose(r["Q_all"][0], (dd ** 2).sum(0), rtol=1e-13, atol=1e-15)
    assert np.allclose(r["S_nt"][0], dd[~tie].sum(0), rtol=1e-13, atol=1e-15)
    mean, se = orc.mc_estimate([node], n, r["S_all"], r["Q_all"], r["paths"])
    assert np.allclose(mean[0], x0 + dd.mean(0), rtol=1e-13)
    assert np.allclose(se[0], dd.std(0, ddof=1) / math.sqrt(60), rtol=1e-9)


def test_step_cap_projects_to_the_nearest_side(orc):
    n = 9
    E = orc.bmap_tables(n, W.BMAP_IDENTITY)
    r = orc.mc_nodes(n, [(4, 4), (1, 4)], E, W.FAMILY_BUMPS, W.COEF_W, (0.0,), seed=1,
                     paths=100, dt=1e-6, max_steps=3)
    assert list(r["non_exits"]) == [100, 100]
    assert list(r["steps"]) == [300, 300]
    pr = orc.path(n, 0.125, 0.5, 0, 0, E, W.FAMILY_BUMPS, W.COEF_W, (0.0,), 1, 1e-6, 3)
    assert pr["capped"] and pr["F"][0] == 0.0          # nearest side is s = 0
    assert abs(pr["F"][1] - 0.5) < 1e-2

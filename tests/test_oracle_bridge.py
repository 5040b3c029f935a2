"""Pins of the oracle's Brownian-bridge exit test (§2.2, the conditional exit
probability of a Brownian bridge, after Gobet): the crossing probability of
the pinned sqrt(2) W against a direct simulation of the bridge, the rule's
edge cases, and its effect: the exit-time and score biases drop from
O(sqrt(dt)) to O(dt)."""
import math

import numpy as np
import pytest

import workloads as W


def test_crossing_probability_matches_simulated_bridges():
    """P(a bridge of sqrt(2) W from a to b over dt dips below 0) =
    exp(-a b / dt), checked against 20000 bridges sampled on 4000 sub-steps
    (first-order correction of the fine grid's own discrete monitoring)."""
    rng = np.random.default_rng(11)
    dt, M = 1e-3, 4000
    for a, b in ((0.02, 0.03), (0.01, 0.05), (0.04, 0.04)):
        p_formula = math.exp(-a * b / dt)
        t = np.arange(1, M + 1) / M
        hits = 0
        K = 20000
        for chunk in range(4):
            inc = rng.normal(0.0, math.sqrt(2 * dt / M), size=(K // 4, M))
            w = np.cumsum(inc, axis=1)
            bridge = a + (b - a) * t + (w - t * w[:, -1:])
            hits += int((bridge.min(axis=1) <= 0.0).sum())
        p_sim = hits / K
        d = 0.5826 * math.sqrt(2 * dt / M)          # fine-grid monitoring shift
        p_fine = math.exp(-(a + d) * (b + d) / dt)
        se = math.sqrt(p_fine * (1 - p_fine) / K)
        assert abs(p_sim - p_fine) < 4 * se + 2e-3, (a, b, p_sim, p_fine, p_formula)


def test_bridge_rule_cases(orc):
    # far from every side: never crosses, no uniforms needed
    assert orc.bridge_exit(0.5, 0.5, 0.51, 0.49, 1e-4, 1, 0, 0, 0)[0] == -1
    # right on the side x and y: p = 1, always crosses that side
    edge, e, tie = orc.bridge_exit(0.3, 1e-300, 0.35, 1e-300, 1e-4, 1, 0, 0, 0)
    assert edge == 0 and e[1] == 0.0 and e[0] == pytest.approx(0.325)
    # the crossing frequency over many counters matches exp(-d0 d1 / dt)
    dt, d0, d1 = 1e-4, 0.004, 0.005
    p = math.exp(-d0 * d1 / dt)
    hits = sum(orc.bridge_exit(d0, 0.5, d1, 0.5, dt, 3, 0, q, 7)[0] == 2 for q in range(20000))
    assert abs(hits / 20000 - p) < 4 * math.sqrt(p * (1 - p) / 20000)


def test_bridge_near_a_corner_tests_each_side_with_its_own_chance(orc):
    """Near the corner (0, 0) two sides can be crossed.  Side s = 0 is tested
    first, then, if it was not crossed, t = 0, each with its own uniform: the
    frequencies must be p_s and (1 - p_s) p_t (one uniform for both sides
    would give max(0, p_t - p_s) for t = 0)."""
    dt = 1e-4
    xs, ys, xt, yt = 0.004, 0.006, 0.003, 0.005
    ps, pt = math.exp(-xs * ys / dt), math.exp(-xt * yt / dt)
    K = 40000
    edges = [orc.bridge_exit(xs, xt, ys, yt, dt, 5, 1, q, 13)[0] for q in range(K)]
    fs = edges.count(2) / K                          # side s = 0 is edge 2
    ft = edges.count(0) / K                          # side t = 0 is edge 0
    want_t = (1 - ps) * pt
    assert abs(fs - ps) < 4 * math.sqrt(ps * (1 - ps) / K), (fs, ps)
    assert abs(ft - want_t) < 4 * math.sqrt(want_t * (1 - want_t) / K), (ft, want_t)
    assert abs(ft - max(0.0, pt - ps)) > 10 * math.sqrt(want_t / K)   # the two rules differ here


def _tau(orc, s0, t0, dt, N, exit_test, seed=9):
    E = orc.bmap_tables(5, W.BMAP_IDENTITY)
    r = orc.mc_nodes(5, [(int(round(s0 * 4)), int(round(t0 * 4)))], E, W.FAMILY_BUMPS, W.COEF_W,
                     (0.0,), seed=seed, paths=N, dt=dt, max_steps=10 ** 6, exit_test=exit_test)
    return float(r["steps"][0]) * dt / N


@pytest.mark.parametrize("s0,t0", [(0.5, 0.5), (0.25, 0.5)])
def test_bridge_removes_the_exit_time_bias(orc, s0, t0):
    """c = 1: E[tau] = torsion function.  At dt = 2e-4 the end-of-step test
    overestimates it by ~0.58 sqrt(2 dt) per side (about 5%), the bridge test
    leaves an O(dt) bias."""
    dt, N = 2e-4, 8000
    v = orc.torsion_exit_time(s0, t0)
    sd = 0.7 * v / math.sqrt(N)                 # std of tau is below 0.7 E[tau] here
    plain = _tau(orc, s0, t0, dt, N, 0)
    bridge = _tau(orc, s0, t0, dt, N, 1)
    assert abs(bridge - v) < 4 * sd + dt, (bridge, v, sd)
    assert plain - v > 6 * sd, (plain, v, sd)


def test_bridge_keeps_the_identity_unbiased_and_sharpens_the_1d_form(orc):
    n = 33
    fam, cm, p = W.FAMILY_BUMPS, W.COEF_W, W.bumps((6.0, 0.35, 0.0, 40.0, 0.0))
    phi = lambda x: orc.closed_form_1d(fam, cm, p, x, axis=0)
    x = np.arange(n) / (n - 1.0)
    E = np.zeros((2, 4, n))
    E[0, 0] = phi(x); E[0, 1] = E[0, 0]; E[0, 2] = 0.0; E[0, 3] = 1.0
    E[1, 2] = x; E[1, 3] = x; E[1, 0] = 0.0; E[1, 1] = 1.0
    nodes = orc.interface_nodes(n, 2, 2)[::3]
    dt = 1e-3                                     # a coarse step
    err = {}
    for et in (0, 1):
        r = orc.mc_nodes(n, nodes, E, fam, cm, p, seed=2, paths=4000, dt=dt, max_steps=10 ** 5,
                         exit_test=et)
        mean, se = orc.mc_estimate(nodes, n, r["S_all"], r["Q_all"], r["paths"])
        exact = np.c_[phi(nodes[:, 0] / (n - 1.0)), nodes[:, 1] / (n - 1.0)]
        err[et] = (np.abs(mean - exact) / se).mean()
    assert err[1] < 1.6, err                      # consistent with pure MC noise
    assert err[0] > err[1] + 0.5, err             # the end-of-step test is biased at this dt

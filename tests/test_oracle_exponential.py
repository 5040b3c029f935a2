"""Pins of the oracle's exponential time stepping (§2.2, after Jansons and
Lythe): step lengths with density lambda exp(-lambda h), the Euler-Maruyama
update over each random length, and the boundary test of each step.

The sharpest pin is a closed form the construction never uses: a driftless
sqrt(2) W run for one Exp(lambda) time from distance a of a side reaches the
side with probability exp(-sqrt(lambda) a) (the running maximum of a Levy
process killed at an independent exponential time is exponential, rate
sqrt(lambda) here).  The oracle gets there through a Gaussian step of a random
length, an end-of-step test and a Brownian-bridge test given the length; a
wrong noise scale, a wrong step-length law or a missing bridge test each moves
the frequency far outside its error bar."""
import math

import numpy as np
import pytest

import workloads as W

FLAT = (0.0,)                     # c = 1: no drift


def test_step_lengths_are_unit_exponentials(orc):
    from scipy import stats
    E = np.array([orc.step_lengths(7, 3, q, k) for q in range(4000) for k in range(5)])
    assert E.shape[1] == 4 and E.min() > 0.0
    for col in range(4):
        assert stats.kstest(E[:, col], "expon").pvalue > 1e-3
    assert abs(E.mean() - 1.0) < 4.0 / math.sqrt(E.size)
    # the words of a block are independent of each other, and of the normals
    # drawn from the same counter (a different stream word)
    for a, b in ((0, 1), (1, 2), (2, 3), (0, 3)):
        assert abs(np.corrcoef(E[:, a], E[:, b])[0, 1]) < 4.0 / math.sqrt(len(E))
    Z = np.array([orc.normals(7, 3, q, k) for q in range(4000) for k in range(5)])
    assert abs(np.corrcoef(E[:, 0], Z[:, 0] ** 2)[0, 1]) < 4.0 / math.sqrt(len(E))


@pytest.mark.parametrize("a,lam", [(0.01, 1e4), (0.02, 1e4), (0.05, 1e3)])
def test_one_exponential_step_reaches_a_side_with_the_closed_form_probability(orc, a, lam):
    n, K = 5, 20000
    E = orc.bmap_tables(n, W.BMAP_IDENTITY)
    hits = 0
    for q in range(K):
        r = orc.path(n, a, 0.5, 1, q, E, W.FAMILY_BUMPS, W.COEF_W, FLAT, 5, 1.0 / lam, 1,
                     exit_test=1, stepper=1)
        if not r["capped"]:
            assert r["F"][0] == 0.0                 # left side s = 0 (identity map)
            hits += 1
    p = math.exp(-math.sqrt(lam) * a)
    se = math.sqrt(p * (1 - p) / K)
    assert abs(hits / K - p) < 4 * se, (hits / K, p, se)
    # without the boundary test only the end-of-step exits remain: far fewer
    ends = sum(not orc.path(n, a, 0.5, 1, q, E, W.FAMILY_BUMPS, W.COEF_W, FLAT, 5, 1.0 / lam,
                            1, exit_test=0, stepper=1)["capped"] for q in range(K))
    assert p - ends / K > 10 * se


@pytest.mark.parametrize("s0,t0", [(0.5, 0.5), (0.25, 0.5)])
def test_mean_exit_time_is_the_torsion_function(orc, s0, t0):
    """c = 1: E[tau] solves Lap v = -1.  The exit time is the sum of the
    steps' random lengths; by Wald's identity its mean is E[steps] / lambda.
    With the boundary test the bias is O(1/lambda); unit noise would double
    the exit time."""
    dt, N = 2e-4, 8000
    E = orc.bmap_tables(5, W.BMAP_IDENTITY)
    r = orc.mc_nodes(5, [(int(round(s0 * 4)), int(round(t0 * 4)))], E, W.FAMILY_BUMPS,
                     W.COEF_W, FLAT, seed=9, paths=N, dt=dt, max_steps=10 ** 6, exit_test=1,
                     stepper=1)
    tau = float(r["steps"][0]) * dt / N
    v = orc.torsion_exit_time(s0, t0)
    sd = 0.7 * v / math.sqrt(N)
    assert abs(tau - v) < 4 * sd + dt, (tau, v, sd)
    assert abs(2 * v - tau) > 20 * sd


def test_exponential_steps_reach_the_one_dimensional_closed_form(orc):
    """c = c(s) at the paper's lambda = 1000: estimates consistent with pure
    Monte Carlo noise around u1 = phi(s), u2 = t; the same mean step without
    any boundary test is visibly biased."""
    n = 33
    fam, cm, p = W.FAMILY_BUMPS, W.COEF_W, W.bumps((6.0, 0.35, 0.0, 40.0, 0.0))
    phi = lambda x: orc.closed_form_1d(fam, cm, p, x, axis=0)
    x = np.arange(n) / (n - 1.0)
    E = np.zeros((2, 4, n))
    E[0, 0] = phi(x); E[0, 1] = E[0, 0]; E[0, 2] = 0.0; E[0, 3] = 1.0
    E[1, 2] = x; E[1, 3] = x; E[1, 0] = 0.0; E[1, 1] = 1.0
    nodes = orc.interface_nodes(n, 2, 2)[::3]
    err = {}
    for et in (0, 1):
        r = orc.mc_nodes(n, nodes, E, fam, cm, p, seed=2, paths=4000, dt=1e-3,
                         max_steps=10 ** 5, exit_test=et, stepper=1)
        mean, se = orc.mc_estimate(nodes, n, r["S_all"], r["Q_all"], r["paths"])
        exact = np.c_[phi(nodes[:, 0] / (n - 1.0)), nodes[:, 1] / (n - 1.0)]
        err[et] = (np.abs(mean - exact) / se).mean()
    assert err[1] < 1.6, err
    assert err[0] > err[1] + 0.5, err


def test_identity_is_unbiased(orc):
    n = 17
    E = orc.bmap_tables(n, W.BMAP_IDENTITY)
    nodes = orc.interface_nodes(n, 2, 2)[::2]
    r = orc.mc_nodes(n, nodes, E, W.FAMILY_BUMPS, W.COEF_W, FLAT, seed=4, paths=3000, dt=1e-3,
                     max_steps=10 ** 5, exit_test=1, stepper=1)
    mean, se = orc.mc_estimate(nodes, n, r["S_all"], r["Q_all"], r["paths"])
    z = (mean - nodes / (n - 1.0)) / se
    assert np.abs(z).max() < 4.0
    assert abs(z.mean()) < 4.0 / math.sqrt(z.size)


def test_node_sums_replay_single_paths(orc):
    n = 9
    E = orc.bmap_tables(n, W.BMAP_IDENTITY)
    p = W.bumps((4.0, 0.4, 0.6, 20.0, 20.0))
    r = orc.mc_nodes(n, [(4, 2)], E, W.FAMILY_BUMPS, W.COEF_INV_W, p, seed=3, paths=50,
                     dt=1e-3, max_steps=10 ** 5, exit_test=1, stepper=1, node_ids=[11])
    S = np.zeros(2)
    steps = 0
    for q in range(50):
        one = orc.path(n, 0.5, 0.25, 11, q, E, W.FAMILY_BUMPS, W.COEF_INV_W, p, 3, 1e-3, 10 ** 5,
                       exit_test=1, stepper=1)
        S += one["F"] - np.array([0.5, 0.25])
        steps += one["steps"]
    assert np.allclose(r["S_all"][0], S, rtol=0, atol=1e-13)
    assert int(r["steps"][0]) == steps

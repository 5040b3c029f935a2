"""Pins of the oracle's Perona-Malik mesh smoothing (§3.4, eq.
PeronaMalikDiffusion, FTCS): the heat-equation limit against the exact decay
of a discrete eigenfunction, fixed points, edge preservation, conservation
and the maximum principle."""
import math

import numpy as np
import pytest


def _grid(n):
    x = np.arange(n) / (n - 1.0)
    return np.meshgrid(x, x, indexing="xy")          # S[j, i] = s_i, T[j, i] = t_j


@pytest.mark.parametrize("p,q,steps,r", [(2, 3, 7, 0.2), (1, 1, 5, 0.25), (5, 2, 3, 0.1)])
def test_heat_limit_decays_a_discrete_eigenfunction_exactly(orc, p, q, steps, r):
    """k -> infinity: g = 1 and each step is u + r Lap_h u, r = dt/h^2.  The
    grid function sin(p pi s) sin(q pi t) is an eigenvector of the five-point
    Laplacian with zero boundary values: every step multiplies it by
    1 - 4 r (sin^2(p pi h/2) + sin^2(q pi h/2))."""
    n = 33
    h = 1.0 / (n - 1)
    S, T = _grid(n)
    U = np.zeros((n, n, 2))
    U[..., 0] = np.sin(p * math.pi * S) * np.sin(q * math.pi * T)
    U[..., 1] = np.sin(q * math.pi * S) * np.sin(p * math.pi * T)
    V = orc.perona_malik(U, steps, r * h * h, 1e12)
    f = 1.0 - 4.0 * r * (math.sin(p * math.pi * h / 2) ** 2 + math.sin(q * math.pi * h / 2) ** 2)
    assert np.max(np.abs(V - f ** steps * U)) < 1e-13


def test_affine_meshes_are_fixed_points(orc):
    """Equal and opposite differences on both sides of every node: an affine
    map is not changed, whatever k."""
    n = 21
    S, T = _grid(n)
    U = np.zeros((n, n, 2))
    U[..., 0] = 0.7 * S + 0.2 * T + 0.05
    U[..., 1] = -0.1 * S + 0.9 * T + 0.1
    for k in (0.3, 1.0, 1000.0):
        V = orc.perona_malik(U, 4, 1e-4, k)
        assert np.max(np.abs(V - U)) < 1e-15


def test_small_k_preserves_an_edge_and_large_k_diffuses_it(orc):
    n = 33
    S, _ = _grid(n)
    U = np.zeros((n, n, 2))
    U[..., 0] = (S >= 0.5).astype(float)               # jump of 1 across one column
    U[..., 1] = U[..., 0]
    dt = 0.2 / (n - 1) ** 2
    kept = orc.perona_malik(U, 3, dt, 1.0)             # |du|/h = 32: g = e^-1024 = 0
    assert np.array_equal(kept, U)
    smoothed = orc.perona_malik(U, 3, dt, 1000.0)
    assert np.max(np.abs(smoothed - U)) > 0.1


def test_conservation_and_maximum_principle(orc):
    """Interior edge fluxes cancel in pairs (the conductance belongs to the
    edge): the interior sum changes only by the flux through the edges to
    the fixed boundary nodes.  With r <= 1/4 no value leaves the range of the
    previous step's values."""
    n = 17
    rng = np.random.default_rng(3)
    S, T = _grid(n)
    U = np.stack([S, T], axis=-1) + 0.02 * rng.standard_normal((n, n, 2))
    h = 1.0 / (n - 1)
    dt, k = 0.25 * h * h, 2.0
    V = orc.perona_malik(U, 1, dt, k)
    r = dt / (h * h)
    for c in range(2):
        u = U[..., c]
        through = 0.0
        for m in range(1, n - 1):
            for (a, b) in (((m, 1), (m, 0)), ((m, n - 2), (m, n - 1)),
                           ((1, m), (0, m)), ((n - 2, m), (n - 1, m))):
                d = u[b] - u[a]
                through += math.exp(-(d / h) ** 2 / (k * k)) * d
        change = (V[1:-1, 1:-1, c] - u[1:-1, 1:-1]).sum()
        assert change == pytest.approx(r * through, rel=1e-10, abs=1e-14)
        assert V[..., c].max() <= u.max() + 1e-15 and V[..., c].min() >= u.min() - 1e-15
    # smoothing lowers the discrete Dirichlet energy of the noise
    def energy(W):
        return sum(float((np.diff(W[..., c], axis=a) ** 2).sum()) for c in range(2) for a in range(2))
    assert energy(orc.perona_malik(U, 5, dt, k)) < energy(U)


def test_zero_steps_is_the_identity(orc):
    U = np.random.default_rng(0).random((9, 9, 2))
    assert np.array_equal(orc.perona_malik(U, 0, 1e-4, 1.0), U)


# ------------------------------------------ smoothing on each subdomain ----
def _noisy(n, seed=3, amp=0.02):
    rng = np.random.default_rng(seed)
    S, T = _grid(n)
    U = np.stack([S, T], axis=-1)
    U[1:-1, 1:-1] += amp * rng.standard_normal((n - 2, n - 2, 2))
    return U


def test_smoothing_lines(orc):
    """Interface lines of the split plus the boundary; shifted, the midlines of
    the blocks those lines bound (each original interface inside a block)."""
    assert orc.smoothing_lines(17, 2, False) == [0, 8, 16]
    assert orc.smoothing_lines(17, 2, True) == [0, 4, 12, 16]
    assert orc.smoothing_lines(29, 3, False) == [0, 9, 19, 28]      # round(28/3), round(56/3)
    assert orc.smoothing_lines(29, 3, True) == [0, 4, 14, 23, 28]
    assert orc.smoothing_lines(17, 1, False) == [0, 16]
    assert orc.smoothing_lines(17, 1, True) == [0, 8, 16]
    for n, s in ((29, 3), (65, 7), (33, 4)):
        X = orc.smoothing_lines(n, s, False)
        Xs = orc.smoothing_lines(n, s, True)
        for a in range(1, len(X) - 1):             # every interface strictly inside a block
            assert any(Xs[b] < X[a] < Xs[b + 1] for b in range(len(Xs) - 1))


def test_one_subdomain_is_the_global_smoothing(orc):
    U = _noisy(21)
    h = 1.0 / 20
    want = orc.perona_malik(U, 4, 0.2 * h * h, 0.7)
    assert np.array_equal(orc.perona_malik_subdomains(U, 4, 0.2 * h * h, 0.7, 1, 1), want)


@pytest.mark.parametrize("sx,sy,shifted", [(2, 2, False), (3, 2, False), (2, 3, True), (4, 4, True)])
def test_blocks_equal_global_steps_with_the_lines_held(orc, sx, sy, shifted):
    """The blocks share only their rings, so smoothing them one by one equals
    smoothing the whole mesh one step at a time with every node on a
    smoothing line put back after each step; the lines are unchanged, and in
    the shifted cycle the original interfaces move."""
    n, steps, k = 29, 5, 0.6
    h = 1.0 / (n - 1)
    dt = 0.22 * h * h
    U = _noisy(n)
    X = orc.smoothing_lines(n, sx, shifted)
    Y = orc.smoothing_lines(n, sy, shifted)
    held = np.zeros((n, n), dtype=bool)
    held[:, X] = True
    held[Y, :] = True
    V = U.copy()
    for _ in range(steps):
        V = orc.perona_malik(V, 1, dt, k)
        V[held] = U[held]
    got = orc.perona_malik_subdomains(U, steps, dt, k, sx, sy, shifted)
    assert np.max(np.abs(got - V)) < 1e-15
    assert np.array_equal(got[held], U[held])
    assert np.all(got[~held] != U[~held])
    if shifted:                                     # the original interfaces are smoothed
        ix = orc.interface_indices(n, sx)
        moved = ~held[1:-1, ix]
        assert moved.mean() > 0.5 and np.all(got[1:-1, ix][moved] != U[1:-1, ix][moved])


@pytest.mark.parametrize("p,q", [(1, 1), (2, 3)])
def test_each_block_decays_with_its_own_eigenvalue(orc, p, q):
    """Heat limit on a 2 x 2 split of n = 33 (blocks of 16 cells): a sine mode
    of each block, zero on the block's ring, decays by 1 - 4 r (sin^2(p pi /
    32) + sin^2(q pi / 32)) per step, the block's own eigenvalue with the
    whole grid's spacing; modes of different blocks do not mix."""
    n, steps, r = 33, 6, 0.2
    h = 1.0 / (n - 1)
    i = np.arange(n)
    U = np.zeros((n, n, 2))
    amp = {(0, 0): 1.0, (1, 0): -0.5, (0, 1): 0.25, (1, 1): 2.0}
    for (a, b), c in amp.items():
        si = np.where((i >= 16 * a) & (i <= 16 * (a + 1)), np.sin(p * math.pi * (i - 16 * a) / 16), 0)
        sj = np.where((i >= 16 * b) & (i <= 16 * (b + 1)), np.sin(q * math.pi * (i - 16 * b) / 16), 0)
        U[..., 0] += c * np.outer(sj, si)
        U[..., 1] += c * np.outer(si, sj)
    got = orc.perona_malik_subdomains(U, steps, r * h * h, 1e12, 2, 2)
    f = 1.0 - 4.0 * r * (math.sin(p * math.pi / 32) ** 2 + math.sin(q * math.pi / 32) ** 2)
    assert np.max(np.abs(got - f ** steps * U)) < 1e-13

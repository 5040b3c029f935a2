"""Pins of the oracle's finite-difference part: the single-domain reference
mesh (§3.2), the 1D boundary forms (§3.2), and the non-iterative domain
decomposition with Dirichlet interface data (§2.1, Fig. 1; §3.5)."""
import numpy as np
import pytest

import workloads as W

BUMP = W.bumps((5.0, 0.5, 0.5, 50.0, 50.0))
BUMP_1D_S = W.bumps((6.0, 0.35, 0.0, 40.0, 0.0))      # c = c(s)
RIDGE_1D_T = (12.0, 60.0, 0.6, 0.0, 1.0)                # a = 0: c = c(t)


def test_constant_coefficient_reproduces_identity(orc):
    """c = 1 with the identity boundary map: u = (s, t) exactly, since linear
    functions satisfy the discrete Laplace equation (§2.1 harmonic maps)."""
    n = 17
    E = orc.bmap_tables(n, W.BMAP_IDENTITY)
    U = orc.global_solve(n, E, W.FAMILY_BUMPS, W.COEF_W, (0.0,))
    x = np.arange(n) / (n - 1.0)
    assert np.max(np.abs(U[:, :, 0] - x[None, :])) < 1e-13
    assert np.max(np.abs(U[:, :, 1] - x[:, None])) < 1e-13


@pytest.mark.parametrize("coef_mode", [W.COEF_W, W.COEF_INV_W])
def test_one_dimensional_coefficient_is_exact(orc, coef_mode):
    """c = c(s) with the paper's boundary map: the 2D discrete solution is the
    discrete 1D solution u1_ij = U_i (from the bottom-edge table) and u2 = t_j."""
    n = 19
    E = orc.bmap_tables(n, W.BMAP_PAPER_1D, W.FAMILY_BUMPS, coef_mode, BUMP_1D_S)
    # the two tables that carry the 1D solution coincide when c = c(s)
    assert np.allclose(E[0, 0], E[0, 1], atol=0, rtol=0)
    U = orc.global_solve(n, E, W.FAMILY_BUMPS, coef_mode, BUMP_1D_S)
    assert np.max(np.abs(U[:, :, 0] - E[0, 0][None, :])) < 1e-13
    t = np.arange(n) / (n - 1.0)
    assert np.max(np.abs(U[:, :, 1] - t[:, None])) < 1e-13
    # and the discrete 1D solution approximates the closed form to O(h^2)
    s = np.arange(n) / (n - 1.0)
    exact = orc.closed_form_1d(W.FAMILY_BUMPS, coef_mode, BUMP_1D_S, s, axis=0)
    assert np.max(np.abs(E[0, 0] - exact)) < 2e-2
    n2 = 2 * n - 1
    E2 = orc.bmap_tables(n2, W.BMAP_PAPER_1D, W.FAMILY_BUMPS, coef_mode, BUMP_1D_S)
    exact2 = orc.closed_form_1d(W.FAMILY_BUMPS, coef_mode, BUMP_1D_S,
                                np.arange(n2) / (n2 - 1.0), axis=0)
    e1 = np.max(np.abs(E[0, 0] - exact))
    e2 = np.max(np.abs(E2[0, 0] - exact2))
    assert 3.0 < e1 / e2 < 5.0            # second order


def test_one_dimensional_in_t(orc):
    n = 15
    E = orc.bmap_tables(n, W.BMAP_PAPER_1D, W.FAMILY_RIDGE, W.COEF_W, RIDGE_1D_T)
    U = orc.global_solve(n, E, W.FAMILY_RIDGE, W.COEF_W, RIDGE_1D_T)
    s = np.arange(n) / (n - 1.0)
    assert np.max(np.abs(U[:, :, 0] - s[None, :])) < 1e-13
    assert np.max(np.abs(U[:, :, 1] - E[1, 2][:, None])) < 1e-13


@pytest.mark.parametrize("n,sx,sy", [(33, 2, 2), (29, 3, 4), (21, 1, 3)])
def test_domain_decomposition_is_exact_with_exact_interface_data(orc, n, sx, sy):
    """Interface values taken from the single-domain solution, then one
    independent Dirichlet solve per subdomain, give back the single-domain
    solution (non-iterative DD, §2.1)."""
    E = orc.bmap_tables(n, W.BMAP_PAPER_1D, W.FAMILY_BUMPS, W.COEF_W, BUMP)
    G = orc.global_solve(n, E, W.FAMILY_BUMPS, W.COEF_W, BUMP)
    nodes = orc.interface_nodes(n, sx, sy)
    iface = G[nodes[:, 1], nodes[:, 0], :]
    S = orc.stitch(n, sx, sy, E, iface, W.FAMILY_BUMPS, W.COEF_W, BUMP)
    assert np.max(np.abs(S - G)) < 1e-12
    # perturbed interface data changes the mesh, by no more than the
    # perturbation (discrete maximum principle)
    S2 = orc.stitch(n, sx, sy, E, iface + 1e-3, W.FAMILY_BUMPS, W.COEF_W, BUMP)
    d = np.max(np.abs(S2 - G))
    assert 1e-4 < d <= 1e-3 + 1e-12


def test_symmetry_about_the_midline(orc):
    """c symmetric about s = 1/2 and the identity map: u1(s) + u1(1-s) = 1."""
    n = 21
    p = W.bumps((9.0, 0.5, 0.3, 30.0, 30.0))
    E = orc.bmap_tables(n, W.BMAP_IDENTITY)
    U = orc.global_solve(n, E, W.FAMILY_BUMPS, W.COEF_W, p)
    assert np.max(np.abs(U[:, :, 0] + U[:, ::-1, 0] - 1.0)) < 1e-12
    assert np.max(np.abs(U[:, :, 1] - U[:, ::-1, 1])) < 1e-12


def test_solution_satisfies_the_stencil_and_maximum_principle(orc):
    n = 25
    fam, p = W.FAMILY_RING, (10.0, 0.5, 0.5, 20.0, 0.25)
    E = orc.bmap_tables(n, W.BMAP_IDENTITY)
    U = orc.global_solve(n, E, fam, W.COEF_W, p)
    cx, cy = orc.edge_coefs(n, fam, W.COEF_W, p)
    assert np.max(np.abs(orc.residual(U, cx, cy))) < 1e-12
    assert U.min() >= -1e-15 and U.max() <= 1 + 1e-15
    # the mesh is adapted: it differs from the identity
    x = np.arange(n) / (n - 1.0)
    assert np.max(np.abs(U[:, :, 0] - x[None, :])) > 1e-2


def test_direct_solve_matches_brute_force_gauss_seidel(orc):
    """Tiny grid: scipy's sparse direct solve against a plain point
    Gauss-Seidel iteration of the stencil run to a fixed point."""
    n = 8
    fam, p = W.FAMILY_BUMPS, W.bumps((4.0, 0.4, 0.6, 20.0, 20.0))
    E = orc.bmap_tables(n, W.BMAP_PAPER_1D, fam, W.COEF_INV_W, p)
    G = orc.global_solve(n, E, fam, W.COEF_INV_W, p)
    cx, cy = orc.edge_coefs(n, fam, W.COEF_INV_W, p)
    U = orc.boundary_grid(n, E)
    for _ in range(3000):
        for j in range(1, n - 1):
            for i in range(1, n - 1):
                cE, cW, cN, cS = cx[j, i], cx[j, i - 1], cy[j, i], cy[j - 1, i]
                U[j, i] = (cE * U[j, i + 1] + cW * U[j, i - 1] + cN * U[j + 1, i]
                           + cS * U[j - 1, i]) / (cE + cW + cN + cS)
    assert np.max(np.abs(U - G)) < 1e-13


def test_torsion_series_matches_a_poisson_solve(orc):
    """The sine series of the mean exit time (Lap v = -1, v = 0 on the
    boundary) against an independent five-point Poisson solve, extrapolated
    in h (Richardson) to remove the O(h^2) error."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    def fd_center(m):
        h = 1.0 / (m + 1)
        e = np.ones(m)
        T = sp.diags([-e[:-1], 2 * e, -e[:-1]], [-1, 0, 1]) / (h * h)
        A = sp.kronsum(T, T).tocsc()
        v = spla.spsolve(A, np.ones(m * m))
        return v.reshape(m, m)[m // 2, m // 2]

    v1, v2 = fd_center(63), fd_center(127)
    extrap = v2 + (v2 - v1) / 3.0
    series = orc.torsion_exit_time(0.5, 0.5)
    assert abs(series - extrap) < 2e-6, (series, extrap)
    assert abs(series - 0.0736713) < 1e-6
    # off-centre value and symmetry
    assert orc.torsion_exit_time(0.25, 0.5) == pytest.approx(orc.torsion_exit_time(0.5, 0.25))
    assert orc.torsion_exit_time(0.0, 0.3) == pytest.approx(0.0, abs=1e-15)

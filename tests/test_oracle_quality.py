"""Pins of the oracle's mesh-quality measures (eq. Qmeasure, §3.1; l_inf,
§3.3) and of the few-point interface (placement and interpolation, §3.6)."""
import math

import numpy as np
import pytest

import workloads as W


def _affine(n, A, b=(0.0, 0.0)):
    x = np.arange(n) / (n - 1.0)
    S, T = np.meshgrid(x, x, indexing="xy")
    U = np.zeros((n, n, 2))
    U[..., 0] = A[0][0] * S + A[0][1] * T + b[0]
    U[..., 1] = A[1][0] * S + A[1][1] * T + b[1]
    return U


def test_quality_of_affine_maps_is_the_singular_value_ratio(orc):
    # Q = (s1^2 + s2^2) / (2 s1 s2) for a linear map with singular values s1, s2
    for A in ([[1, 0], [0, 1]], [[0.5, 0], [0, 0.8]], [[0.6, 0.2], [-0.1, 0.7]]):
        U = _affine(9, A)
        s = np.linalg.svd(np.array(A, dtype=float), compute_uv=False)
        want = (s[0] ** 2 + s[1] ** 2) / (2 * s[0] * s[1])
        q = orc.cell_quality(U)
        assert np.allclose(q, want, rtol=1e-12)
    assert np.all(orc.cell_quality(_affine(5, [[1, 0], [0, 1]])) == 1.0)


def test_quality_is_at_least_one_and_detects_folds(orc):
    spec = W.config1()
    E = orc.bmap_tables(spec.n, 0)
    G = orc.global_solve(spec.n, E, spec.family, spec.coef_mode, spec.params)
    q = orc.cell_quality(G)
    assert np.all(q >= 1.0 - 1e-14) and np.isfinite(q).all()
    F = G.copy()
    F[10, 10], F[10, 11] = G[10, 11].copy(), G[10, 10].copy()     # swap two nodes
    res = orc.mesh_quality(F)
    assert res["folds"] >= 1


def test_ratios_and_l_inf(orc):
    spec = W.config1()
    E = orc.bmap_tables(spec.n, 0)
    G = orc.global_solve(spec.n, E, spec.family, spec.coef_mode, spec.params)
    same = orc.mesh_quality(G, G, spec.family, spec.coef_mode, spec.params)
    assert same["r_max"] == 1.0 and same["r_mean"] == 1.0 and same["l_inf"] == 0.0
    # moving one node by delta changes w there by about |grad w| delta
    H = G.copy()
    H[16, 10, 0] += 1e-3
    res = orc.mesh_quality(H, G, spec.family, spec.coef_mode, spec.params)
    gw = abs(orc.coef(spec.family, 0, spec.params, H[16, 10, 0], H[16, 10, 1])
             - orc.coef(spec.family, 0, spec.params, G[16, 10, 0], G[16, 10, 1]))
    assert res["l_inf"] == pytest.approx(gw, rel=1e-12)
    assert res["r_max"] <= 1.0 + 1e-12


def test_extrema_placement_matches_the_closed_form(orc):
    """rho = 1 + A exp(-k (t - 1/2)^2) along a vertical line: rho' has its
    extrema at 1/2 +- 1/sqrt(2k), rho'' at 1/2 and 1/2 +- sqrt(3/(2k))."""
    n, k = 257, 60.0
    p = W.bumps((5.0, 0.5, 0.5, 0.0, k))          # depends on t only
    mask = orc.placement(n, 2, 1, 2, family=W.FAMILY_BUMPS, params=p)
    nodes = orc.interface_nodes(n, 2, 1)[mask]
    t = np.sort(nodes[:, 1]) / (n - 1.0)
    want = np.sort([0.5 - 1 / math.sqrt(2 * k), 0.5 + 1 / math.sqrt(2 * k), 0.5,
                    0.5 - math.sqrt(1.5 / k), 0.5 + math.sqrt(1.5 / k)])
    assert len(t) == 5
    assert np.max(np.abs(t - want)) <= 1.0 / (n - 1)


def test_equispaced_placement_and_crossings(orc):
    mask = orc.placement(33, 2, 2, 1, k=7)
    nodes = orc.interface_nodes(33, 2, 2)[mask]
    assert len(nodes) == 13                          # 7 + 7 - the shared crossing
    assert (16, 16) in {tuple(x) for x in nodes}
    # a flat density has no extrema: only the crossing remains
    m2 = orc.placement(33, 2, 2, 2, family=W.FAMILY_BUMPS, params=(0.0,))
    assert m2.sum() == 1


def test_interpolation_is_exact_for_linear_data(orc):
    n, sx, sy = 33, 3, 2
    E = orc.bmap_tables(n, 0)
    nodes = orc.interface_nodes(n, sx, sy)
    exact = nodes / (n - 1.0)                        # identity: linear along every line
    mask = orc.placement(n, sx, sy, 1, k=3)
    vals = np.where(mask[:, None], exact, 123.0)
    got = orc.interpolate_interface(n, sx, sy, E, mask, vals)
    assert np.allclose(got, exact, atol=1e-15)
    assert np.array_equal(got[mask], exact[mask])

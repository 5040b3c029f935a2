"""The fully probabilistic mesh (§3.3: Monte Carlo at every interior node)
and Perona-Malik smoothing (§3.4) on the GPU, against the oracle."""
from dataclasses import replace

import numpy as np
import pytest

import workloads as W
from gpu_helpers import gpu_plan

pytestmark = pytest.mark.gpu


def _noisy_mesh(n, seed=0, amp=0.01):
    rng = np.random.default_rng(seed)
    x = np.arange(n) / (n - 1.0)
    S, T = np.meshgrid(x, x, indexing="xy")
    U = np.stack([S, T], axis=-1)
    U[1:-1, 1:-1] += amp * rng.standard_normal((n - 2, n - 2, 2))
    return U


@pytest.mark.parametrize("steps", [1, 2, 5, 10])
@pytest.mark.parametrize("k", [1000.0, 0.5])
def test_smoothing_matches_oracle(orc, steps, k):
    import torch
    from paper_1310_3435_gb300 import native as N
    spec = W.small_parity_cases()[0]
    n = spec.n
    h = 1.0 / (n - 1)
    dt = 0.2 * h * h
    U = _noisy_mesh(n)
    want = orc.perona_malik(U, steps, dt, k)
    with gpu_plan(spec) as P:
        host = U.copy()
        N.sdd_mesh_smooth(P.handle, host, steps, dt, k)
        assert np.max(np.abs(host - want)) < 1e-13
        dev = torch.from_numpy(U.copy()).cuda()
        N.sdd_mesh_smooth(P.handle, dev, steps, dt, k)
        torch.cuda.synchronize()
        assert np.array_equal(dev.cpu().numpy(), host)
    # the boundary is untouched and the noise is damped
    assert np.array_equal(host[0], U[0]) and np.array_equal(host[:, -1], U[:, -1])


@pytest.mark.parametrize("sx,sy,shifted,steps", [(2, 2, False, 5), (3, 2, False, 1), (2, 3, True, 5),
                                                  (4, 4, True, 2), (1, 1, True, 3), (5, 7, False, 10)])
def test_subdomain_smoothing_matches_oracle(orc, sx, sy, shifted, steps):
    """Smoothing on each subdomain (interface lines held) and on the shifted
    subdomains, host and device meshes, against the oracle's block-by-block
    smoothing; the held lines stay bitwise unchanged."""
    import torch
    from paper_1310_3435_gb300 import native as N
    n, k = 29, 0.6
    spec = W.MeshSpec(n=n, sx=sx, sy=sy, family=W.FAMILY_BUMPS,
                      params=W.bumps((5.0, 0.5, 0.5, 50.0, 50.0)), paths=8, dt=1e-4, seed=1)
    dt = 0.22 / (n - 1) ** 2
    U = _noisy_mesh(n, seed=sx * 10 + sy)
    want = orc.perona_malik_subdomains(U, steps, dt, k, sx, sy, shifted)
    with gpu_plan(spec) as P:
        host = U.copy()
        N.sdd_mesh_smooth_subdomains(P.handle, host, steps, dt, k, shifted)
        dev = torch.from_numpy(U.copy()).cuda()
        N.sdd_mesh_smooth_subdomains(P.handle, dev, steps, dt, k, shifted)
        torch.cuda.synchronize()
        assert np.array_equal(dev.cpu().numpy(), host)
    assert np.max(np.abs(host - want)) < 1e-13
    X = orc.smoothing_lines(n, sx, shifted)
    Y = orc.smoothing_lines(n, sy, shifted)
    assert np.array_equal(host[:, X], U[:, X]) and np.array_equal(host[Y, :], U[Y, :])


def test_smoothing_validation():
    from paper_1310_3435_gb300 import native as N
    spec = W.small_parity_cases()[0]
    n = spec.n
    U = _noisy_mesh(n)
    with gpu_plan(spec) as P:
        same = U.copy()
        N.sdd_mesh_smooth(P.handle, same, 0, 1e-4, 1.0)
        assert np.array_equal(same, U)
        with pytest.raises(N.SddError):
            N.sdd_mesh_smooth(P.handle, U.copy(), 3, 0.3 / (n - 1) ** 2, 1.0)   # r > 1/4
        with pytest.raises(N.SddError):
            N.sdd_mesh_smooth(P.handle, U.copy(), -1, 1e-5, 1.0)
        with pytest.raises(N.SddError):
            N.sdd_mesh_smooth(P.handle, U.copy(), 1, 1e-5, 0.0)
        with pytest.raises(N.SddError):
            load = N.load()
            rc = load.sdd_mesh_smooth_subdomains(P.handle, N._ptr(U.copy()), 1, 1e-5, 1.0, 2, None)
            N._check(rc, "sdd_mesh_smooth_subdomains")
        with pytest.raises(N.SddError):
            N.sdd_mesh_smooth_subdomains(P.handle, U.copy(), 3, 0.3 / (n - 1) ** 2, 1.0, True)


def test_fully_probabilistic_mesh_matches_oracle(orc):
    """sx = sy = n - 1: every interior node is a Monte Carlo node; the mesh is
    the boundary map on the boundary and the node estimates inside."""
    from paper_1310_3435_gb300 import native as N
    spec = replace(W.small_parity_cases()[3], sx=12, sy=12, paths=600,
                   stepper=W.STEP_EXPONENTIAL, exit_test=W.EXIT_BRIDGE, dt=1e-3)
    n = spec.n
    with gpu_plan(spec) as P:
        assert P.n_nodes == (n - 2) ** 2
        nodes = P.nodes()
        mesh = np.zeros((n, n, 2))
        mean = np.zeros((P.n_nodes, 2))
        ms, ss = N.sdd_mesh_generate(P.handle, P.mc_params(), P.solve_params(), mesh, mean)
        assert ss.subdomains == (n - 1) ** 2 and ss.converged == ss.subdomains
    assert set(map(tuple, nodes)) == {(i, j) for i in range(1, n - 1) for j in range(1, n - 1)}
    E = orc.bmap_tables(n, spec.bmap_mode, spec.family, spec.coef_mode, spec.params)
    o = orc.mc_nodes(n, nodes, E, spec.family, spec.coef_mode, spec.params, seed=spec.seed,
                     paths=spec.paths, dt=spec.dt, max_steps=spec.cap(), tie_delta=spec.tie(),
                     exit_test=spec.exit_test, stepper=spec.stepper)
    assert int(o["ties"].sum()) == 0
    mo, _ = orc.mc_estimate(nodes, n, o["S_all"], o["Q_all"], o["paths"])
    assert np.max(np.abs(mean - mo) / np.abs(mo)) < 1e-11
    assert np.array_equal(mesh[nodes[:, 1], nodes[:, 0]], mean)
    B = orc.boundary_grid(n, E)
    ring = np.ones((n, n), bool)
    ring[1:-1, 1:-1] = False
    assert np.array_equal(mesh[ring], B[ring])


def test_smoothing_improves_a_noisy_probabilistic_mesh(orc):
    """The paper's observation (§3.4): a few Perona-Malik steps bring the
    quality of a low-N fully probabilistic mesh of the running example
    towards the deterministic mesh's."""
    import math
    from paper_1310_3435_gb300 import native as N
    rho = W.bumps((15.0 * math.exp(-0.5), 0.75, 0.5, 50.0, 50.0))
    spec = W.MeshSpec(n=29, sx=28, sy=28, family=W.FAMILY_BUMPS, params=rho,
                      coef_mode=W.COEF_INV_W, bmap_mode=W.BMAP_PAPER_1D, paths=1000, dt=1e-3,
                      precision=W.FP32_STEP, stepper=W.STEP_EXPONENTIAL, exit_test=W.EXIT_BRIDGE)
    E = orc.bmap_tables(29, spec.bmap_mode, spec.family, spec.coef_mode, rho)
    ref = orc.global_solve(29, E, spec.family, spec.coef_mode, rho)
    with gpu_plan(spec) as P:
        mesh = np.zeros((29, 29, 2))
        N.sdd_mesh_generate(P.handle, P.mc_params(), P.solve_params(), mesh)
        q0 = N.sdd_mesh_quality(P.handle, mesh, ref)
        sm = mesh.copy()
        N.sdd_mesh_smooth(P.handle, sm, 10, 1e-4, 1000.0)
        q1 = N.sdd_mesh_quality(P.handle, sm, ref)
    assert q1["q_max"] < q0["q_max"] and q1["l_inf"] < q0["l_inf"]
    assert abs(q1["r_max"] - 1.0) < abs(q0["r_max"] - 1.0)


def test_smoothing_and_fully_probabilistic_edge_cases(orc):
    """n = 3: one interior node, one smoothing stencil; the fully
    probabilistic plan has that one node."""
    from paper_1310_3435_gb300 import native as N
    spec = W.MeshSpec(n=3, sx=2, sy=2, family=W.FAMILY_BUMPS,
                      params=W.bumps((4.0, 0.4, 0.6, 20.0, 20.0)), paths=64, dt=1e-3)
    U = _noisy_mesh(3, seed=5, amp=0.05)
    dt = 0.25 * 0.25                                  # h = 1/2: r = dt/h^2 = 1/4 exactly
    want = orc.perona_malik(U, 3, dt, 0.7)
    with gpu_plan(spec) as P:
        assert P.n_nodes == 1
        got = U.copy()
        N.sdd_mesh_smooth(P.handle, got, 3, dt, 0.7)
    assert np.max(np.abs(got - want)) < 1e-15

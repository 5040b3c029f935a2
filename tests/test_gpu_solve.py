"""Parity of the CUDA subdomain solves and of the whole mesh generation with
the oracle (§2.1, Fig. 1; §3.2; §3.5).  Meshes agree to 1e-10 when both
sides solve to near rounding level."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import gpu_means, gpu_plan, gpu_sums, oracle_edges, oracle_sums

pytestmark = pytest.mark.gpu

MESH_TOL = 1e-10


def _solve(spec, iface, solver, tol, max_iter=0):
    from paper_1310_3435_gb300 import native as N
    with gpu_plan(spec) as P:
        mesh = np.zeros((spec.n, spec.n, 2))
        st = N.sdd_subdomain_solve(P.handle, np.ascontiguousarray(iface, dtype=np.float64),
                                   N.solve_params(solver=solver, tol=tol, max_iter=max_iter), mesh)
        return mesh, st


CASES = [
    W.config1(),
    W.MeshSpec(n=29, sx=3, sy=4, family=W.FAMILY_RING, params=(10.0, 0.5, 0.5, 20.0, 0.25)),
    W.MeshSpec(n=41, sx=2, sy=3, family=W.FAMILY_RIDGE, params=(20.0, 200.0, 0.3, 0.2, 1.0),
               coef_mode=W.COEF_INV_W, bmap_mode=W.BMAP_PAPER_1D),
    W.MeshSpec(n=65, sx=2, sy=2, family=W.FAMILY_BUMPS,
               params=W.bumps((8.0, 0.3, 0.6, 30.0, 10.0), (3.0, 0.7, 0.2, 80.0, 80.0))),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("solver", [W.SOLVER_SOR, W.SOLVER_CG_FP32_REFINE,
                                    W.SOLVER_CG_JACOBI_FP32_REFINE])
def test_domain_decomposition_exactness(orc, case, solver):
    """Interface data from the oracle's single-domain mesh: the GPU stitched
    mesh reproduces that mesh (non-iterative DD is exact with exact data)."""
    spec = CASES[case]
    E = oracle_edges(orc, spec)
    G = orc.global_solve(spec.n, E, spec.family, spec.coef_mode, spec.params)
    nodes = orc.interface_nodes(spec.n, spec.sx, spec.sy)
    iface = G[nodes[:, 1], nodes[:, 0], :]
    mesh, st = _solve(spec, iface, solver, 1e-13)
    assert st.converged == st.subdomains
    assert np.max(np.abs(mesh - G)) <= MESH_TOL


@pytest.mark.parametrize("solver", [W.SOLVER_SOR, W.SOLVER_CG_FP32_REFINE,
                                    W.SOLVER_CG_JACOBI_FP32_REFINE])
def test_solve_matches_oracle_with_noisy_interface(orc, solver):
    """Interface values with Monte Carlo-like noise: the stitched meshes of
    both sides agree (the solve is linear in the Dirichlet data)."""
    spec = CASES[1]
    nodes = orc.interface_nodes(spec.n, spec.sx, spec.sy)
    rng = np.random.default_rng(3)
    iface = nodes / (spec.n - 1.0) + rng.normal(0, 5e-3, size=nodes.shape)
    E = oracle_edges(orc, spec)
    ref = orc.stitch(spec.n, spec.sx, spec.sy, E, iface, spec.family, spec.coef_mode, spec.params)
    mesh, st = _solve(spec, iface, solver, 1e-13)
    assert np.max(np.abs(mesh - ref)) <= MESH_TOL


def test_multigrid_preconditioner_cuts_the_iterations(orc):
    """197 x 197 split 2 x 2 (97 x 97 interior nodes per subdomain, the
    paper's four-subdomain case, where the solves dominate): the multigrid-
    preconditioned CG needs a few dozen iterations in all, the diagonally
    preconditioned one hundreds; both match the oracle's stitched mesh."""
    spec = W.MeshSpec(n=197, sx=2, sy=2, family=W.FAMILY_RING,
                      params=(10.0, 0.5, 0.5, 50.0, 0.25))
    nodes = orc.interface_nodes(spec.n, spec.sx, spec.sy)
    rng = np.random.default_rng(5)
    iface = nodes / (spec.n - 1.0) + rng.normal(0, 2e-3, size=nodes.shape)
    ref = orc.stitch(spec.n, spec.sx, spec.sy, oracle_edges(orc, spec), iface, spec.family,
                     spec.coef_mode, spec.params)
    mesh_mg, st_mg = _solve(spec, iface, W.SOLVER_CG_FP32_REFINE, 1e-13)
    mesh_j, st_j = _solve(spec, iface, W.SOLVER_CG_JACOBI_FP32_REFINE, 1e-13)
    assert st_mg.converged == st_j.converged == 4
    assert st_mg.max_iterations <= 60, st_mg.max_iterations
    assert st_j.max_iterations >= 5 * st_mg.max_iterations, (st_j.max_iterations,
                                                            st_mg.max_iterations)
    assert st_mg.node_iterations <= 4 * 97 * 97 * st_mg.max_iterations
    assert np.max(np.abs(mesh_mg - ref)) <= MESH_TOL
    assert np.max(np.abs(mesh_j - ref)) <= MESH_TOL


def test_solver_tolerance_and_stats(orc):
    spec = CASES[3]
    nodes = orc.interface_nodes(spec.n, spec.sx, spec.sy)
    E = oracle_edges(orc, spec)
    G = orc.global_solve(spec.n, E, spec.family, spec.coef_mode, spec.params)
    iface = G[nodes[:, 1], nodes[:, 0], :]
    for solver in (W.SOLVER_SOR, W.SOLVER_CG_FP32_REFINE, W.SOLVER_CG_JACOBI_FP32_REFINE):
        mesh, st = _solve(spec, iface, solver, 1e-10)
        assert st.converged == st.subdomains == 4
        assert st.max_rel_residual <= 1e-10
        assert st.max_iterations > 0
    # an iteration cap too small to converge is reported
    from paper_1310_3435_gb300 import native as N
    with gpu_plan(spec) as P:
        mesh = np.zeros((spec.n, spec.n, 2))
        with pytest.raises(N.SddError) as e:
            N.sdd_subdomain_solve(P.handle, iface, N.solve_params(W.SOLVER_SOR, 1e-12, 8), mesh)
        assert e.value.code == N.SDD_ERR_NOT_CONVERGED


def test_mesh_generate_config1_matches_oracle(orc):
    """Whole pipeline on the plain-FP64 configuration (33x33, 2x2, N=4000):
    GPU mesh vs the oracle's stitched mesh built from the oracle's own
    interface estimates."""
    from paper_1310_3435_gb300 import native as N
    spec = W.config1()
    nodes = orc.interface_nodes(spec.n, spec.sx, spec.sy)
    o = oracle_sums(orc, spec)
    mo, _ = orc.mc_estimate(nodes, spec.n, o["S_all"], o["Q_all"], o["paths"])
    E = oracle_edges(orc, spec)
    ref = orc.stitch(spec.n, spec.sx, spec.sy, E, mo, spec.family, spec.coef_mode, spec.params)
    with gpu_plan(spec) as P:
        mesh = np.zeros((spec.n, spec.n, 2))
        im = np.zeros((P.n_nodes, 2))
        ise = np.zeros((P.n_nodes, 2))
        ms, ss = N.sdd_mesh_generate(P.handle, P.mc_params(), P.solve_params(tol=1e-13), mesh,
                                     im, ise)
    assert int(o["ties"].sum()) == 0 and ms.ties == 0
    assert np.max(np.abs(im - mo)) <= 1e-12
    assert np.max(np.abs(mesh - ref)) <= MESH_TOL
    assert ss.converged == ss.subdomains
    assert ms.path_steps == int(o["steps"].sum())
    # the mesh is a valid adapted mesh: inside the square, not the identity
    assert mesh.min() >= 0 and mesh.max() <= 1


def test_whole_domain_when_unsplit(orc):
    """1 x 1 split: no interface, one subdomain = the single-domain solve."""
    spec = W.MeshSpec(n=25, sx=1, sy=1, family=W.FAMILY_BUMPS, params=W.bumps((5.0, .5, .5, 50, 50)))
    E = oracle_edges(orc, spec)
    G = orc.global_solve(spec.n, E, spec.family, spec.coef_mode, spec.params)
    mesh, st = _solve(spec, np.zeros((0, 2)), W.SOLVER_SOR, 1e-13)
    assert np.max(np.abs(mesh - G)) <= MESH_TOL

"""Few-point interfaces (§3.6: placement, Monte Carlo at the placed nodes,
interpolation) and the mesh-quality measures (§3.1, §3.3) on the GPU, against
the oracle."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import gpu_plan, oracle_edges

pytestmark = pytest.mark.gpu

CASES = [
    (W.config1(paths=600), W.EXIT_END_OF_STEP),
    (W.MeshSpec(n=41, sx=3, sy=2, family=W.FAMILY_RING, params=(10.0, 0.5, 0.5, 30.0, 0.25),
                paths=500, dt=1e-4, seed=3), W.EXIT_BRIDGE),
]


@pytest.mark.parametrize("mode,k", [(1, 7), (2, 0)])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_placement_and_interpolation_match_oracle(orc, mode, k, case):
    from paper_1310_3435_gb300 import native as N
    spec, et = CASES[case]
    spec = W.MeshSpec(**{**spec.__dict__, "exit_test": et})
    want = orc.placement(spec.n, spec.sx, spec.sy, mode, k=k, family=spec.family,
                         params=spec.params)
    with gpu_plan(spec) as P:
        full = np.zeros((P.n_nodes, 2))
        N.sdd_interface_mc(P.handle, P.mc_params(), full, None)
        N.sdd_plan_set_placement(P.handle, mode, k)
        mask, n_mc = N.sdd_plan_placement(P.handle)
        assert np.array_equal(mask, want) and n_mc == int(want.sum())
        few = np.zeros((P.n_nodes, 2))
        se = np.zeros((P.n_nodes, 2))
        st = N.sdd_interface_mc(P.handle, P.mc_params(), few, se)
        assert st.paths == spec.paths * n_mc
    # Monte Carlo nodes: the same estimates as the full run (same streams)
    assert np.allclose(few[mask], full[mask], rtol=1e-13, atol=0)
    # the others: interpolated along their line, as the oracle does
    E = oracle_edges(orc, spec)
    ref = orc.interpolate_interface(spec.n, spec.sx, spec.sy, E, mask, full)
    assert np.allclose(few, ref, rtol=0, atol=1e-13)


def test_few_point_mesh_generation_and_batch(orc):
    from paper_1310_3435_gb300 import native as N
    import torch
    spec = CASES[0][0]
    with gpu_plan(spec) as P, gpu_plan(spec) as Q:
        N.sdd_plan_set_placement(P.handle, N.SDD_PLACE_EXTREMA, 0)
        N.sdd_plan_set_placement(Q.handle, N.SDD_PLACE_EXTREMA, 0)
        mesh = np.zeros((spec.n, spec.n, 2))
        N.sdd_mesh_generate(P.handle, P.mc_params(), P.solve_params(tol=1e-12), mesh)
        stream = torch.cuda.Stream()
        with N.Batch([Q], [Q.mc_params()], [Q.solve_params(tol=1e-12)]) as B:
            B.run(stream=stream)
            stream.synchronize()
            mb = np.zeros((spec.n, spec.n, 2))
            N.sdd_plan_results(Q.handle, mb)
        assert np.array_equal(mesh, mb)


def test_quality_matches_oracle(orc):
    from paper_1310_3435_gb300 import native as N
    spec = W.config1()
    E = oracle_edges(orc, spec)
    G = orc.global_solve(spec.n, E, spec.family, spec.coef_mode, spec.params)
    rng = np.random.default_rng(0)
    H = G.copy()
    H[1:-1, 1:-1] += rng.normal(0, 2e-3, size=H[1:-1, 1:-1].shape)
    with gpu_plan(spec) as P:
        for mesh, ref in ((G, None), (H, G)):
            got = N.sdd_mesh_quality(P.handle, np.ascontiguousarray(mesh),
                                     None if ref is None else np.ascontiguousarray(ref))
            want = orc.mesh_quality(mesh, ref, spec.family, spec.coef_mode, spec.params)
            assert got["q_max"] == pytest.approx(want["q_max"], rel=1e-12)
            assert got["q_mean"] == pytest.approx(want["q_mean"], rel=1e-10)
            assert got["folds"] == want["folds"]
            if ref is not None:
                assert got["r_max"] == pytest.approx(want["r_max"], rel=1e-12)
                assert got["r_mean"] == pytest.approx(want["r_mean"], rel=1e-10)
                assert got["l_inf"] == pytest.approx(want["l_inf"], rel=1e-12)
        F = G.copy()
        F[10, 10], F[10, 11] = G[10, 11].copy(), G[10, 10].copy()
        assert N.sdd_mesh_quality(P.handle, F)["folds"] == orc.mesh_quality(F)["folds"] > 0

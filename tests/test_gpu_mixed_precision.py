"""The mixed-precision product as the bench, the batches and the server run
it: interface values from FP32 stepping with FP64 sums (§2.2), then FP32 CG
inside FP64 iterative refinement on every subdomain (§2.1, Fig. 1; §3.5).

* Against the oracle's stitched mesh on the same interface values, the mesh
  must lie within 1e-6 in mesh coordinates (the solves' share of the error).
* Against the mesh the oracle stitches from its own FP64 interface values on
  the same Philox streams, it must lie within the largest interface
  difference (plus that 1e-6): the subdomain solves obey a discrete maximum
  principle, so interface differences reach the mesh without growth.  That
  interface difference is the precision-induced bias, within half a standard
  error at every node.
* The largest workload, 1025 x 1025 split 8 x 8 with the anisotropic ridge:
  sampled nodes against the FP64 oracle on the same streams."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import gpu_means, gpu_plan, oracle_edges

pytestmark = pytest.mark.gpu

MESH_BOUND = 1e-6


def _generate(spec):
    """Mesh, interface means and std-errs of one mixed-precision generation."""
    from paper_1310_3435_gb300 import native as N
    with gpu_plan(spec) as P:
        mesh = np.zeros((spec.n, spec.n, 2))
        mean = np.zeros((P.n_nodes, 2))
        se = np.zeros((P.n_nodes, 2))
        ms, ss = N.sdd_mesh_generate(P.handle, P.mc_params(), P.solve_params(), mesh, mean, se)
    assert ss.converged == ss.subdomains
    return mesh, mean, se


def _stitch(orc, spec, iface):
    return orc.stitch(spec.n, spec.sx, spec.sy, oracle_edges(orc, spec), iface, spec.family,
                      spec.coef_mode, spec.params)


def test_bench_workload_mesh_within_1e6_of_the_oracle_stitch(orc):
    """257 x 257, 4 x 4, ring, N = 1e5, dt = 1e-5, as the bench times it."""
    spec = W.config2()
    assert spec.precision == W.FP32_STEP and spec.solver == W.SOLVER_CG_FP32_REFINE
    mesh, mean, _ = _generate(spec)
    ref = _stitch(orc, spec, mean)
    err = float(np.abs(mesh - ref).max())
    assert err <= MESH_BOUND, err


def test_batched_meshes_within_1e6_of_the_oracle_stitch(orc):
    """Eight meshes of the batched workload (n in {65..513}, splits 2..8,
    N = 2e4, dt = 5e-5) generated as one batch."""
    import torch
    from paper_1310_3435_gb300 import native as N
    specs = W.config3(count=8)
    plans = [gpu_plan(s) for s in specs]
    stream = torch.cuda.Stream()
    with N.Batch(plans) as B:
        B.run(use_graph=True, stream=stream)
        stream.synchronize()
        for i, (s, P) in enumerate(zip(specs, plans)):
            mesh = np.zeros((s.n, s.n, 2))
            mean = np.zeros((P.n_nodes, 2))
            N.sdd_plan_results(P.handle, mesh, mean, None)
            _, ss = B.stats(i)
            assert ss.converged == ss.subdomains, s.label
            err = float(np.abs(mesh - _stitch(orc, s, mean)).max())
            assert err <= MESH_BOUND, (s.label, err)
    for P in plans:
        P.close()


@pytest.mark.parametrize("spec", [
    W.config2(paths=128),
    [s for s in W.config3(count=16) if s.n == 65][0],
], ids=["ring257", "batched65"])
def test_mixed_precision_mesh_against_the_fp64_oracle_mesh(orc, spec):
    """Reduced N (the oracle runs every interface node on the same streams)."""
    if spec.n == 65:
        spec = W.MeshSpec(**{**spec.__dict__, "paths": 512})
    mesh, mean, se = _generate(spec)
    nodes = orc.interface_nodes(spec.n, spec.sx, spec.sy)
    o = orc.mc_nodes(spec.n, nodes, oracle_edges(orc, spec), spec.family, spec.coef_mode,
                     spec.params, seed=spec.seed, paths=spec.paths, dt=spec.dt,
                     max_steps=spec.cap(), tie_delta=1e-11)
    mo, so = orc.mc_estimate(nodes, spec.n, o["S_all"], o["Q_all"], o["paths"])
    bias = np.abs(mean - mo)
    assert np.all(bias <= 0.5 * so + 1e-15), float((bias / so).max())
    assert float(np.abs(mesh - _stitch(orc, spec, mean)).max()) <= MESH_BOUND
    bound = float(bias.max()) + MESH_BOUND
    err = float(np.abs(mesh - _stitch(orc, spec, mo)).max())
    assert err <= bound, (err, bound)


def test_precision_stress_workload_on_sampled_nodes(orc):
    """1025 x 1025, 8 x 8, ridge w = 1 + 20 exp(-200 (t - 0.3 - 0.2 sin 2 pi s)^2),
    dt = 1e-5, FP32 stepping, in the bench's launch configuration (one
    single-mesh launch over all 14273 nodes), 4096 paths per node: 32 evenly
    spaced nodes against the FP64 oracle on the same streams, within half a
    standard error, step counts within 1e-3."""
    from paper_1310_3435_gb300 import native as N
    spec = W.config4(paths=4096)
    with gpu_plan(spec) as P:
        assert P.n_nodes == 14273
        g = N.sdd_interface_mc_sums(P.handle, P.mc_params())
        nodes = P.nodes()
    idx = (np.arange(32) * (len(nodes) // 32)).astype(int)
    o = orc.mc_nodes(spec.n, nodes[idx], oracle_edges(orc, spec), spec.family, spec.coef_mode,
                     spec.params, seed=spec.seed, paths=spec.paths, dt=spec.dt,
                     max_steps=spec.cap(), tie_delta=1e-11, node_ids=idx)
    mo, so = orc.mc_estimate(nodes[idx], spec.n, o["S_all"], o["Q_all"], o["paths"])
    mg, _ = gpu_means(g[idx], spec.n, nodes[idx])
    assert np.all(np.abs(mg - mo) <= 0.5 * so), float((np.abs(mg - mo) / so).max())
    assert np.array_equal(g["paths"][idx], o["paths"])
    steps_o = int(o["steps"].sum())
    assert abs(int(g["steps"][idx].sum()) - steps_o) / steps_o < 1e-3

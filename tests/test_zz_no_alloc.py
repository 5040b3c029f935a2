"""The allocation-free Monte Carlo entry point, for callers that cannot
allocate device memory (their allocator belongs to someone else, or an
allocation would synchronise or fail at that point).  It must give the same
interface estimates as the plan-based entry point, on two calls in a row,
since all calls share one static scratch array that keeps the last call's
contents.  This file is collected last, so a run that stops at the first
failure has run every other test before it."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _inputs(spec):
    import torch
    from paper_1310_3435_gb300 import native as N
    with N.Plan(spec) as P:
        nodes = torch.from_numpy(P.nodes()).cuda()
        edges = torch.from_numpy(np.ascontiguousarray(P.edges())).cuda()
        mean = np.zeros((P.n_nodes, 2))
        se = np.zeros((P.n_nodes, 2))
        N.sdd_interface_mc(P.handle, P.mc_params(chunk=256), mean, se)
        return nodes, edges, mean, se, P.density


@pytest.mark.parametrize("spec", [
    W.config1(paths=1000),                                               # FP64 stepping
    W.MeshSpec(n=41, sx=3, sy=2, family=W.FAMILY_RING, params=(10.0, 0.5, 0.5, 50.0, 0.25),
               paths=777, dt=1e-4, seed=9, precision=W.FP32_STEP),
    W.MeshSpec(n=37, sx=2, sy=3, family=W.FAMILY_RIDGE, params=(20.0, 200.0, 0.3, 0.2, 1.0),
               paths=640, dt=1e-4, seed=5, precision=W.FP32_STEP, stepper=W.STEP_EXPONENTIAL,
               exit_test=W.EXIT_BRIDGE),                                 # the paper's stepper
])
def test_static_scratch_matches_the_plan_entry_point_twice(spec):
    import torch
    from paper_1310_3435_gb300 import native as N
    nodes, edges, mean_ref, se_ref, dens = _inputs(spec)
    mc = N.mc_params(spec.paths, spec.dt, spec.seed, spec.precision, chunk=256,
                     max_steps=spec.max_steps, tie_delta=spec.tie_delta,
                     exit_test=spec.exit_test, stepper=spec.stepper)
    stream = torch.cuda.Stream()
    for _ in range(2):                               # the scratch keeps the last call's data
        mean = torch.full((nodes.shape[0], 2), -1.0, dtype=torch.float64, device="cuda")
        se = torch.full((nodes.shape[0], 2), -1.0, dtype=torch.float64, device="cuda")
        N.sdd_interface_mc_static(spec.n, nodes, edges, dens, mc, mean, se, stream=stream)
        stream.synchronize()
        assert np.allclose(mean.cpu().numpy(), mean_ref, rtol=1e-12, atol=0)
        assert np.allclose(se.cpu().numpy(), se_ref, rtol=1e-12, atol=0)


def test_static_scratch_rejects_work_beyond_its_size():
    import torch
    from paper_1310_3435_gb300 import native as N
    spec = W.config2(paths=4 * 10 ** 8)             # 1521 nodes x ceil(4e8 / 8192) items
    nodes = torch.zeros((1521, 2), dtype=torch.int32, device="cuda")
    edges = torch.zeros((2, 4, spec.n), dtype=torch.float64, device="cuda")
    mean = torch.zeros((1521, 2), dtype=torch.float64, device="cuda")
    dens = N.make_density(spec.family, spec.params)
    with pytest.raises(N.SddError) as e:
        N.sdd_interface_mc_static(spec.n, nodes, edges, dens, N.mc_params(spec.paths, spec.dt),
                                  mean)
    assert e.value.code == N.SDD_ERR_INVALID_ARG
    assert "static scratch" in N.sdd_last_error()

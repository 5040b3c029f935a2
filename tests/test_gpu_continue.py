"""A run that continues a plan's previous run (sdd_mc_params.path_begin): the
estimator is a sum over paths (§2.2; §6 notes the additivity of the
expectation), so the paths of a first, shorter run (a pilot) count in the
final estimate.  The continued run must give bitwise the result of one run of
N paths with the same work-item size, alone and inside a batch, and must
refuse to continue a run it cannot."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import gpu_plan

pytestmark = pytest.mark.gpu

CASES = [
    W.MeshSpec(n=41, sx=3, sy=2, family=W.FAMILY_RING, params=(10.0, 0.5, 0.5, 50.0, 0.25),
               paths=1500, dt=1e-4, seed=9, precision=W.FP32_STEP),
    W.config1(paths=1100),                                             # FP64 stepping
    W.MeshSpec(n=37, sx=2, sy=3, family=W.FAMILY_RIDGE, params=(20.0, 200.0, 0.3, 0.2, 1.0),
               paths=999, dt=1e-4, seed=5, precision=W.FP32_STEP, stepper=W.STEP_EXPONENTIAL,
               exit_test=W.EXIT_BRIDGE),
]
CHUNK = 256
PILOT = 512


def _whole(spec):
    """One run of all N paths (chunk CHUNK): sums, mean, stderr, stats."""
    from paper_1310_3435_gb300 import native as N
    with gpu_plan(spec) as P:
        mc = P.mc_params(chunk=CHUNK)
        mean = np.zeros((P.n_nodes, 2))
        se = np.zeros((P.n_nodes, 2))
        st = N.sdd_interface_mc(P.handle, mc, mean, se)
        sums = N.sdd_interface_mc_sums(P.handle, mc)
        return sums, mean, se, st


@pytest.mark.parametrize("case", range(len(CASES)))
def test_continued_run_is_bitwise_one_run(case):
    from paper_1310_3435_gb300 import native as N
    spec = CASES[case]
    sums_ref, mean_ref, se_ref, st_ref = _whole(spec)
    with gpu_plan(spec) as P:
        pilot = P.mc_params(paths=PILOT, chunk=CHUNK)
        ps = N.sdd_interface_mc(P.handle, pilot, np.zeros((P.n_nodes, 2)), None)
        assert ps.paths == PILOT * P.n_nodes
        mc = P.mc_params(chunk=CHUNK, path_begin=PILOT)
        mean = np.zeros((P.n_nodes, 2))
        se = np.zeros((P.n_nodes, 2))
        st = N.sdd_interface_mc(P.handle, mc, mean, se)
        assert np.array_equal(mean, mean_ref)
        assert np.array_equal(se, se_ref)
        assert (st.paths, st.path_steps, st.ties, st.non_exits) == (
            st_ref.paths, st_ref.path_steps, st_ref.ties, st_ref.non_exits)
        assert st.max_stderr == st_ref.max_stderr
        sums = N.sdd_interface_mc_sums(P.handle, P.mc_params(paths=PILOT, chunk=CHUNK))
        assert np.all(sums["paths"] == PILOT)


def test_continued_run_of_a_ragged_pilot_and_twice():
    """A continued run continues in turn (pilot 512 -> 1024 -> 1500)."""
    from paper_1310_3435_gb300 import native as N
    spec = CASES[0]
    sums_ref, mean_ref, se_ref, _ = _whole(spec)
    with gpu_plan(spec) as P:
        N.sdd_interface_mc(P.handle, P.mc_params(paths=PILOT, chunk=CHUNK), None, None,
                           want_stats=False)
        N.sdd_interface_mc(P.handle, P.mc_params(paths=1024, chunk=CHUNK, path_begin=PILOT),
                           None, None, want_stats=False)
        sums = N.sdd_interface_mc_sums(P.handle, P.mc_params(chunk=CHUNK, path_begin=1024))
    assert sums.tobytes() == sums_ref.tobytes()


def test_continued_runs_in_a_batch_are_bitwise_one_run():
    import torch
    from paper_1310_3435_gb300 import native as N
    specs = [W.MeshSpec(**{**s.__dict__, "solver": W.SOLVER_CG_FP32_REFINE}) for s in CASES]
    specs += W.config3(count=3, seed=5, paths=1300, dt=2e-4)
    ref = []
    for s in specs:
        with gpu_plan(s) as P:
            mesh = np.zeros((s.n, s.n, 2))
            mean = np.zeros((P.n_nodes, 2))
            se = np.zeros((P.n_nodes, 2))
            N.sdd_mesh_generate(P.handle, P.mc_params(chunk=CHUNK), P.solve_params(), mesh, mean,
                                se)
            ref.append((mesh, mean, se))
    plans = [gpu_plan(s) for s in specs]
    for P in plans:                                       # the pilots, each alone
        N.sdd_interface_mc(P.handle, P.mc_params(paths=PILOT, chunk=CHUNK), None, None,
                           want_stats=False)
    mcs = [P.mc_params(chunk=CHUNK, path_begin=PILOT) for P in plans]
    stream = torch.cuda.Stream()
    for use_graph in (False, True):
        with N.Batch(plans, mcs, [P.solve_params() for P in plans]) as B:
            for _ in range(2):
                B.run(use_graph=use_graph, stream=stream)
                stream.synchronize()
                for i, (s, P) in enumerate(zip(specs, plans)):
                    mesh = np.zeros((s.n, s.n, 2))
                    mean = np.zeros((P.n_nodes, 2))
                    se = np.zeros((P.n_nodes, 2))
                    N.sdd_plan_results(P.handle, mesh, mean, se)
                    ms, _ = B.stats(i)
                    assert ms.paths == s.paths * P.n_nodes
                    assert np.array_equal(mean, ref[i][1]), (use_graph, i)
                    assert np.array_equal(se, ref[i][2]), (use_graph, i)
                    assert np.array_equal(mesh, ref[i][0]), (use_graph, i)
    for P in plans:
        P.close()


def test_continuation_is_refused_when_it_cannot_hold():
    from paper_1310_3435_gb300 import native as N
    spec = CASES[0]
    with gpu_plan(spec) as P:
        def refused(mc, what):
            with pytest.raises(N.SddError) as e:
                N.sdd_interface_mc(P.handle, mc, None, None, want_stats=False)
            assert e.value.code == N.SDD_ERR_INVALID_ARG
            assert what in N.sdd_last_error(), N.sdd_last_error()
        refused(P.mc_params(chunk=CHUNK, path_begin=PILOT), "no previous whole run")
        N.sdd_interface_mc(P.handle, P.mc_params(paths=PILOT, chunk=CHUNK), None, None,
                           want_stats=False)
        refused(P.mc_params(chunk=0, path_begin=PILOT), "explicit chunk")
        refused(P.mc_params(chunk=CHUNK, path_begin=PILOT + 32), "divides path_begin")
        refused(P.mc_params(chunk=CHUNK, path_begin=PILOT, seed=spec.seed + 1), "other parameters")
        refused(P.mc_params(chunk=CHUNK, path_begin=PILOT, dt=spec.dt * 2), "other parameters")
        refused(P.mc_params(chunk=2 * CHUNK, path_begin=PILOT), "other parameters")
        refused(P.mc_params(paths=PILOT - CHUNK, chunk=CHUNK, path_begin=PILOT), "must not exceed")
        # a split run overwrites the items: nothing left to continue
        N.sdd_interface_mc_advance(P.handle, P.mc_params(chunk=CHUNK), 1)
        refused(P.mc_params(chunk=CHUNK, path_begin=PILOT), "no previous whole run")
        # a batch whose plan ran another Monte Carlo since the batch was made
        N.sdd_interface_mc(P.handle, P.mc_params(paths=PILOT, chunk=CHUNK), None, None,
                           want_stats=False)
        with N.Batch([P], [P.mc_params(chunk=CHUNK, path_begin=PILOT)], [P.solve_params()]) as B:
            N.sdd_interface_mc(P.handle, P.mc_params(paths=2 * PILOT, chunk=CHUNK), None, None,
                               want_stats=False)
            with pytest.raises(N.SddError) as e:
                B.run()
            assert e.value.code == N.SDD_ERR_INVALID_ARG

"""A Monte Carlo run split over calls and resumed from a checkpoint gives
bitwise the same node estimates as one call (the sums are additive over work
items, and every item's sums do not depend on the launch that ran it)."""
from dataclasses import replace

import numpy as np
import pytest

import workloads as W
from gpu_helpers import gpu_plan

pytestmark = pytest.mark.gpu


def _whole(P, mc):
    from paper_1310_3435_gb300 import native as N
    mean = np.zeros((P.n_nodes, 2))
    se = np.zeros((P.n_nodes, 2))
    st = N.sdd_interface_mc(P.handle, mc, mean, se)
    return mean, se, st


@pytest.mark.parametrize("precision,stepper", [(W.FP32_STEP, W.STEP_EULER),
                                               (W.FP64, W.STEP_EULER),
                                               (W.FP32_STEP, W.STEP_EXPONENTIAL)])
def test_split_run_equals_one_call(precision, stepper):
    from paper_1310_3435_gb300 import native as N
    spec = replace(W.small_parity_cases()[1], precision=precision, stepper=stepper,
                   exit_test=W.EXIT_BRIDGE)
    with gpu_plan(spec) as P:
        mc = P.mc_params(chunk=64)
        want_mean, want_se, want_st = _whole(P, mc)
        done, total = N.sdd_interface_mc_advance(P.handle, mc, 5)
        assert done == 5 and total > 10
        while done < total:
            done, _ = N.sdd_interface_mc_advance(P.handle, mc, 7)
        mean = np.zeros((P.n_nodes, 2))
        se = np.zeros((P.n_nodes, 2))
        st = N.sdd_interface_mc_finish(P.handle, mc, mean, se)
    assert np.array_equal(mean, want_mean) and np.array_equal(se, want_se)
    assert st.path_steps == want_st.path_steps and st.paths == want_st.paths


def test_checkpoint_resumes_on_a_new_plan():
    from paper_1310_3435_gb300 import native as N
    spec = replace(W.small_parity_cases()[2], precision=W.FP32_STEP)
    with gpu_plan(spec) as P:
        mc = P.mc_params(chunk=32)
        want_mean, _, want_st = _whole(P, mc)
        done, total = N.sdd_interface_mc_advance(P.handle, mc, 11)
        blob = N.sdd_mc_checkpoint_save(P.handle)
        with pytest.raises(N.SddError):                     # items are left
            N.sdd_interface_mc_finish(P.handle, mc)
    with gpu_plan(spec) as Q:                               # the first plan is gone
        N.sdd_mc_checkpoint_load(Q.handle, blob)
        while done < total:
            done, _ = N.sdd_interface_mc_advance(Q.handle, mc, 13)
        mean = np.zeros((Q.n_nodes, 2))
        st = N.sdd_interface_mc_finish(Q.handle, mc, mean)
    assert np.array_equal(mean, want_mean) and st.path_steps == want_st.path_steps


def test_checkpoint_is_checked():
    from paper_1310_3435_gb300 import native as N
    spec = replace(W.small_parity_cases()[2], precision=W.FP32_STEP)
    other = replace(spec, seed=spec.seed + 1, params=(21.0,) + tuple(spec.params[1:]))
    with gpu_plan(spec) as P:
        mc = P.mc_params(chunk=32)
        N.sdd_interface_mc_advance(P.handle, mc, 3)
        blob = N.sdd_mc_checkpoint_save(P.handle)
    with gpu_plan(other) as Q:                              # another density
        with pytest.raises(N.SddError):
            N.sdd_mc_checkpoint_load(Q.handle, blob)
    with gpu_plan(spec) as R:
        with pytest.raises(N.SddError):
            N.sdd_mc_checkpoint_load(R.handle, blob[:-8])    # truncated
        with pytest.raises(N.SddError):
            N.sdd_mc_checkpoint_load(R.handle, b"x" * len(blob))

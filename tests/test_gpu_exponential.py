"""Exponential time stepping on the GPU (§2.2, after Jansons and Lythe):
parity of FP64 stepping with the oracle, FP32 stepping paired with FP64,
batches against single-mesh runs, and a sampled check at the 257 x 257 ring
workload."""
from dataclasses import replace

import numpy as np
import pytest

import workloads as W
from gpu_helpers import gpu_means, gpu_plan, gpu_sums

pytestmark = pytest.mark.gpu

# FP64 parity bar of exponential steps.  Their lengths have an exponential
# tail: on the steep ring case (k = 50, mean step 1e-4) a step of several mean
# lengths has h |grad b| > 1, where the explicit Euler-Maruyama update
# amplifies a perturbation several-fold per step.  Perturbing each normal of
# the oracle by one ulp moves that case's per-node means by up to 2.6e-13
# (each step length: 1.5e-13; constant steps: 4e-14 to 8e-14), and the GPU
# differs from the host by an ulp or two in several functions per step
# (log, sincospi, exp).  The bar is 1e-11, about 40 single-ulp sensitivities;
# any error in the method itself shows up at 1e-6 and above.
REL_EXPO = 1e-11


def _expo(spec, exit_test=W.EXIT_BRIDGE, **kw):
    return replace(spec, stepper=W.STEP_EXPONENTIAL, exit_test=exit_test, **kw)


def _oracle(orc, spec, nodes, paths=None, node_ids=None):
    E = orc.bmap_tables(spec.n, spec.bmap_mode, spec.family, spec.coef_mode, spec.params)
    return orc.mc_nodes(spec.n, nodes, E, spec.family, spec.coef_mode, spec.params,
                        seed=spec.seed, paths=paths or spec.paths, dt=spec.dt,
                        max_steps=spec.cap(), tie_delta=spec.tie(), exit_test=spec.exit_test,
                        stepper=spec.stepper, node_ids=node_ids)


@pytest.mark.parametrize("exit_test", [W.EXIT_BRIDGE, W.EXIT_END_OF_STEP])
@pytest.mark.parametrize("case", range(len(W.small_parity_cases())))
def test_fp64_exponential_matches_oracle(orc, case, exit_test):
    spec = _expo(W.small_parity_cases()[case], exit_test)
    nodes = orc.interface_nodes(spec.n, spec.sx, spec.sy)
    g = gpu_sums(spec)
    o = _oracle(orc, spec, nodes)
    n = spec.n
    assert np.array_equal(g["paths"], o["paths"])
    assert np.array_equal(g["non_exits"], o["non_exits"])
    clean = (g["ties"] == 0) & (o["ties"] == 0)
    assert np.array_equal(g["steps"][clean], o["steps"][clean])
    mg, _ = gpu_means(g, n, nodes, nt=True)
    mo, _ = orc.mc_estimate(nodes, n, o["S_nt"], o["Q_nt"], o["paths"] - o["ties"])
    rel = np.abs(mg - mo) / np.maximum(np.abs(mo), 1e-300)
    # how many node components miss the constant-step bar of 1e-12 (reported,
    # not asserted: the bar here is REL_EXPO, see above)
    print("exponential parity %s: %d of %d node components above 1e-12 relative (max %.2e)"
          % (spec.label, int((rel > 1e-12).sum()), rel.size, float(rel.max())))
    assert rel.max() <= REL_EXPO, rel.max()
    # the random steps are not the constant ones
    g_euler = gpu_sums(replace(spec, stepper=W.STEP_EULER))
    assert not np.array_equal(g_euler["steps"], g["steps"])


@pytest.mark.parametrize("case", [0, 1, 2])
def test_fp32_exponential_paired_with_fp64(orc, case):
    spec = _expo(W.small_parity_cases()[case])
    nodes = orc.interface_nodes(spec.n, spec.sx, spec.sy)
    g64 = gpu_sums(spec, precision=W.FP64)
    g32 = gpu_sums(spec, precision=W.FP32_STEP)
    m64, se64 = gpu_means(g64, spec.n, nodes)
    m32, _ = gpu_means(g32, spec.n, nodes)
    # FP32 and FP64 paths share their random numbers but drift apart where
    # long steps meet steep drift (the ring case), so the paired difference is
    # bounded against the Monte Carlo error, not absolutely: at every node at
    # most half a standard error, and no systematic shift on average
    d = np.abs(m32 - m64)
    assert np.all(d <= 0.5 * se64), (d / se64).max()
    assert abs((m32 - m64).mean()) < 0.1 * se64.mean()
    rel_steps = abs(int(g32["steps"].sum()) - int(g64["steps"].sum())) / g64["steps"].sum()
    assert rel_steps < 2e-3
    assert int(g32["non_exits"].sum()) == int(g64["non_exits"].sum()) == 0


def test_batch_equals_single_runs():
    """A batch mixing constant and exponential steps over several density
    classes gives every mesh the same sums as its own single-mesh run."""
    from paper_1310_3435_gb300 import native as N
    specs = [_expo(s, precision=W.FP32_STEP) for s in W.small_parity_cases()[:3]]
    specs.append(replace(W.small_parity_cases()[1], precision=W.FP32_STEP))
    specs.append(_expo(W.small_parity_cases()[0]))                  # FP64, exponential
    plans = [gpu_plan(s) for s in specs]
    try:
        single = []
        for P in plans:
            sums = N.sdd_interface_mc_sums(P.handle, P.mc_params())
            mean = np.zeros((P.n_nodes, 2))
            N.sdd_plan_results(P.handle, None, mean, None)
            single.append((int(sums["steps"].sum()), mean))
        with N.Batch(plans) as B:
            B.run()
            for k, P in enumerate(plans):
                ms, _ = B.stats(k)
                got = np.zeros((P.n_nodes, 2))
                N.sdd_plan_results(P.handle, None, got, None)
                assert np.array_equal(got, single[k][1]), k
                assert int(ms.path_steps) == single[k][0]
    finally:
        for P in plans:
            P.close()


def test_ring_workload_sampled_nodes_match_the_oracle(orc):
    """The 257 x 257 ring workload with exponential steps at the paper's
    lambda = 1e4, FP32 stepping as timed: sampled nodes against the FP64
    oracle on the same streams (paired difference within the FP64 estimate's
    standard error)."""
    spec = _expo(W.config2(paths=2048, dt=1e-4))
    with gpu_plan(spec) as P:
        from paper_1310_3435_gb300 import native as N
        g = N.sdd_interface_mc_sums(P.handle, P.mc_params())
        nodes_all = P.nodes()
    pick = np.arange(0, len(nodes_all), len(nodes_all) // 24)[:24]
    o = _oracle(orc, replace(spec, precision=W.FP64), nodes_all[pick], node_ids=pick)
    mo, seo = orc.mc_estimate(nodes_all[pick], spec.n, o["S_all"], o["Q_all"], o["paths"])
    mg, _ = gpu_means(g[pick], spec.n, nodes_all[pick])
    assert np.all(np.abs(mg - mo) <= seo), (np.abs(mg - mo) / seo).max()
    rel = abs(int(g["steps"][pick].sum()) - int(o["steps"].sum())) / o["steps"].sum()
    assert rel < 2e-3


def test_paper_stepper_at_full_size_matches_the_oracle_on_sampled_nodes(orc):
    """The bench's paper-stepper leg as it is timed: the 257 x 257 ring,
    4 x 4, N = 1e5, exponential steps at lambda = 1e4 with the bridge test,
    FP32 stepping, one single-mesh launch.  Two nodes, one on the ring's
    steep flank and one inside it, against the FP64 oracle on the same 1e5
    Philox streams (run in path ranges over the host cores): the paired
    difference within half a standard error, step counts within 1e-3."""
    from concurrent.futures import ThreadPoolExecutor
    from paper_1310_3435_gb300 import native as N
    spec = _expo(W.config2(dt=1e-4))
    assert spec.paths == 100000
    with gpu_plan(spec) as P:
        g = N.sdd_interface_mc_sums(P.handle, P.mc_params())
        nodes = P.nodes()
    r = np.hypot(nodes[:, 0] / 256.0 - 0.5, nodes[:, 1] / 256.0 - 0.5)
    pick = [int(np.argmin(np.abs(r - 0.27))), int(np.argmin(np.abs(r - 0.12)))]
    E = orc.bmap_tables(spec.n, spec.bmap_mode, spec.family, spec.coef_mode, spec.params)
    parts = 16
    per = spec.paths // parts

    def run(job):
        k, q = job
        return orc.mc_nodes(spec.n, nodes[[k]], E, spec.family, spec.coef_mode, spec.params,
                            seed=spec.seed, paths=per, dt=spec.dt, max_steps=spec.cap(),
                            tie_delta=spec.tie(), node_ids=[k], threads=1, path_begin=q * per,
                            exit_test=spec.exit_test, stepper=spec.stepper)

    jobs = [(k, q) for k in pick for q in range(parts)]
    with ThreadPoolExecutor(max_workers=orc.default_threads()) as ex:
        outs = list(ex.map(run, jobs))
    for a, k in enumerate(pick):
        mine = outs[a * parts:(a + 1) * parts]
        S = sum(o["S_all"][0] for o in mine)
        Q = sum(o["Q_all"][0] for o in mine)
        steps = sum(int(o["steps"][0]) for o in mine)
        mo, so = orc.mc_estimate(nodes[[k]], spec.n, S[None, :], Q[None, :], [spec.paths])
        mg, _ = gpu_means(g[[k]], spec.n, nodes[[k]])
        assert np.all(np.abs(mg - mo) <= 0.5 * so), (k, mg, mo, so)
        assert int(g["paths"][k]) == spec.paths
        assert abs(int(g["steps"][k]) - steps) / steps < 1e-3


def test_unknown_stepper_is_rejected():
    from paper_1310_3435_gb300 import native as N
    spec = W.small_parity_cases()[1]
    with gpu_plan(spec) as P:
        with pytest.raises(N.SddError):
            N.sdd_interface_mc_sums(P.handle, P.mc_params(stepper=7))


def test_exponential_edge_cases(orc):
    """n = 3 (one node), N = 2, and a step cap of 3 that ends most paths:
    counts and capped scores replay the oracle."""
    for cap, et in ((3, W.EXIT_END_OF_STEP), (3, W.EXIT_BRIDGE), (0, W.EXIT_BRIDGE)):
        spec = W.MeshSpec(n=3, sx=2, sy=2, family=W.FAMILY_RING,
                          params=(10.0, 0.5, 0.5, 50.0, 0.25), paths=2, dt=1e-3, seed=7,
                          max_steps=cap, stepper=W.STEP_EXPONENTIAL, exit_test=et)
        nodes = orc.interface_nodes(spec.n, spec.sx, spec.sy)
        g = gpu_sums(spec)
        o = _oracle(orc, spec, nodes)
        assert np.array_equal(g["paths"], o["paths"])
        assert np.array_equal(g["non_exits"], o["non_exits"])
        assert np.array_equal(g["steps"], o["steps"])
        assert np.allclose(g["sum"], o["S_all"], rtol=1e-11, atol=1e-15)

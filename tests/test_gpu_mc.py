"""Parity of the CUDA interface Monte Carlo with the FP64 oracle (§2.2).

FP64 stepping replays the oracle's Philox streams: per node, over the paths
neither side flags as an exit-decision tie, the means agree to 1e-12
relative and the step counts exactly.  FP32 stepping (same streams) is
checked as a paired difference against FP64: its precision bias is stated
separately from the Monte Carlo error."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import gpu_means, gpu_plan, gpu_sums, oracle_sums

pytestmark = pytest.mark.gpu

REL_FP64 = 1e-12


def _compare_fp64(orc, spec, g, o, nodes):
    n = spec.n
    assert np.array_equal(g["paths"], o["paths"])
    assert np.array_equal(g["non_exits"], o["non_exits"])
    ties_g, ties_o = g["ties"].astype(np.int64), o["ties"].astype(np.int64)
    both_clean = (ties_g == 0) & (ties_o == 0)
    # exit decisions identical => identical step counts, bit for bit
    assert np.array_equal(g["steps"][both_clean], o["steps"][both_clean])
    mg, _ = gpu_means(g, n, nodes, nt=True)
    mo, _ = orc.mc_estimate(nodes, n, o["S_nt"], o["Q_nt"], o["paths"] - o["ties"])
    rel = np.abs(mg - mo) / np.maximum(np.abs(mo), 1e-300)
    assert rel.max() <= REL_FP64, (rel.max(), np.unravel_index(rel.argmax(), rel.shape))
    return int(ties_g.sum()), int(ties_o.sum())


@pytest.mark.parametrize("case", range(len(W.small_parity_cases())))
def test_fp64_matches_oracle(orc, case):
    spec = W.small_parity_cases()[case]
    nodes = orc.interface_nodes(spec.n, spec.sx, spec.sy)
    g = gpu_sums(spec)
    o = oracle_sums(orc, spec)
    _compare_fp64(orc, spec, g, o, nodes)


def test_fp64_full_config1_matches_oracle(orc):
    """33x33, 2x2, N = 4000, dt = 1e-4: the plain-FP64 configuration at full
    size, every node."""
    spec = W.config1()
    nodes = orc.interface_nodes(spec.n, spec.sx, spec.sy)
    g = gpu_sums(spec)
    o = oracle_sums(orc, spec)
    tg, to = _compare_fp64(orc, spec, g, o, nodes)
    assert tg == to


def test_plan_matches_oracle_nodes_and_tables(orc):
    from paper_1310_3435_gb300 import native as N
    for spec in W.small_parity_cases() + [W.config1(), W.config2()]:
        with gpu_plan(spec) as P:
            assert np.array_equal(P.nodes(), orc.interface_nodes(spec.n, spec.sx, spec.sy))
            E = orc.bmap_tables(spec.n, spec.bmap_mode, spec.family, spec.coef_mode, spec.params)
            assert np.allclose(P.edges(), E, rtol=0, atol=1e-14)


def test_stats_and_determinism(orc):
    from paper_1310_3435_gb300 import native as N
    spec = W.small_parity_cases()[1]
    with gpu_plan(spec) as P:
        mc = P.mc_params()
        a = N.sdd_interface_mc_sums(P.handle, mc)
        b = N.sdd_interface_mc_sums(P.handle, mc)
        assert a.tobytes() == b.tobytes()              # bitwise reproducible
        st = N.sdd_plan_last_mc_stats(P.handle)
        assert st.paths == spec.paths * P.n_nodes
        assert st.path_steps == int(a["steps"].sum())
        assert st.ties == int(a["ties"].sum())
        # another chunking sums the same paths in another order
        c = N.sdd_interface_mc_sums(P.handle, P.mc_params(chunk=64))
        assert np.array_equal(c["steps"], a["steps"])
        assert np.allclose(c["sum"], a["sum"], rtol=1e-13, atol=1e-13)
        mean = np.zeros((P.n_nodes, 2))
        se = np.zeros((P.n_nodes, 2))
        st2 = N.sdd_interface_mc(P.handle, mc, mean, se)
        m2, s2 = gpu_means(a, spec.n, P.nodes())
        assert np.allclose(mean, m2, rtol=1e-14, atol=0)
        assert np.allclose(se, s2, rtol=1e-12, atol=0)
        assert st2.max_stderr == pytest.approx(s2.max(), rel=1e-12)


def test_device_and_host_outputs_agree():
    import torch
    from paper_1310_3435_gb300 import native as N
    spec = W.config1(paths=512)
    with gpu_plan(spec) as P:
        mc = P.mc_params()
        mh = np.zeros((P.n_nodes, 2))
        N.sdd_interface_mc(P.handle, mc, mh, None)
        md = torch.zeros((P.n_nodes, 2), dtype=torch.float64, device="cuda")
        sd = torch.zeros((P.n_nodes, 2), dtype=torch.float64, device="cuda")
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            N.sdd_interface_mc(P.handle, mc, md, sd, want_stats=False, stream=s)
        s.synchronize()
        assert np.array_equal(md.cpu().numpy(), mh)
        assert (sd > 0).all()


def test_edge_cases(orc):
    from paper_1310_3435_gb300 import native as N
    # smallest grid with an interface node, fewest paths, odd step cap
    spec = W.MeshSpec(n=3, sx=2, sy=2, family=W.FAMILY_BUMPS, params=(0.0,), paths=2,
                      dt=1e-3, seed=1, max_steps=7)
    g = gpu_sums(spec)
    o = oracle_sums(orc, spec)
    assert g.shape == (1,)
    _compare_fp64(orc, spec, g, o, orc.interface_nodes(3, 2, 2))
    # every path capped: 3 steps of size sqrt(2e-7) cannot reach a side from
    # the nearest interface node (distance 1/32)
    spec = W.config1(paths=100, max_steps=3, dt=1e-7)
    g = gpu_sums(spec)
    assert np.all(g["non_exits"] == 100) and np.all(g["steps"] == 300)
    o = oracle_sums(orc, spec)
    _compare_fp64(orc, spec, g, o, orc.interface_nodes(33, 2, 2))
    # no interface at all (1 x 1 split): nothing to do
    spec = W.MeshSpec(n=9, sx=1, sy=1, family=W.FAMILY_BUMPS, params=(0.0,), paths=10)
    with gpu_plan(spec) as P:
        assert P.n_nodes == 0
        st = N.sdd_interface_mc(P.handle, P.mc_params())
        assert st.paths == 0 and st.path_steps == 0
    # invalid Monte Carlo parameters
    with gpu_plan(W.config1()) as P:
        for kw in (dict(paths=1), dict(dt=0.0), dict(precision=5), dict(chunk=33)):
            with pytest.raises(N.SddError) as e:
                N.sdd_interface_mc(P.handle, P.mc_params(**kw))
            assert e.value.code == N.SDD_ERR_INVALID_ARG


@pytest.mark.parametrize("case", [0, 1, 2])
def test_fp32_stepping_paired_with_fp64(orc, case):
    """Same Philox streams in FP32 stepping: the difference to FP64 is the
    precision-induced bias.  It must stay below the Monte Carlo error of the
    estimate and below 1e-3 absolute at every node."""
    spec = W.small_parity_cases()[case]
    nodes = orc.interface_nodes(spec.n, spec.sx, spec.sy)
    g64 = gpu_sums(spec, precision=W.FP64)
    g32 = gpu_sums(spec, precision=W.FP32_STEP)
    m64, se64 = gpu_means(g64, spec.n, nodes)
    m32, se32 = gpu_means(g32, spec.n, nodes)
    d = np.abs(m32 - m64)
    assert d.max() < 1e-3, d.max()
    assert np.all(d <= se64), (d / se64).max()
    # the bias is systematic-free on average: mean paired difference << stderr
    assert abs((m32 - m64).mean()) < 0.1 * se64.mean()
    # step counts differ only through paths whose exit decision moved
    rel_steps = abs(int(g32["steps"].sum()) - int(g64["steps"].sum())) / g64["steps"].sum()
    assert rel_steps < 1e-3


def test_fp32_sums_are_exact_and_reproducible(orc):
    """FP32 stepping accumulates fixed-point sums: bitwise identical across
    runs, and across work-item sizes up to the final FP64 rounding."""
    from paper_1310_3435_gb300 import native as N
    spec = W.small_parity_cases()[1]
    with gpu_plan(spec) as P:
        mc = P.mc_params(precision=W.FP32_STEP)
        a = N.sdd_interface_mc_sums(P.handle, mc)
        b = N.sdd_interface_mc_sums(P.handle, mc)
        assert a.tobytes() == b.tobytes()
        st = N.sdd_plan_last_mc_stats(P.handle)
        assert st.ties == 0 and st.paths == spec.paths * P.n_nodes
        assert np.all(a["paths"] == spec.paths)
        for chunk in (32, 64, 256, 8192):
            c = N.sdd_interface_mc_sums(P.handle, P.mc_params(precision=W.FP32_STEP, chunk=chunk))
            assert np.array_equal(c["steps"], a["steps"])
            assert np.array_equal(c["paths"], a["paths"])
            assert np.allclose(c["sum"], a["sum"], rtol=1e-15, atol=1e-12)
            assert np.allclose(c["sumsq"], a["sumsq"], rtol=1e-15, atol=1e-12)


@pytest.mark.parametrize("case", range(len(W.small_parity_cases())))
def test_fp64_bridge_matches_oracle(orc, case):
    """The Brownian-bridge exit test replays the oracle too (its uniforms come
    from the same Philox streams, counter word 3 = 1)."""
    spec = W.MeshSpec(**{**W.small_parity_cases()[case].__dict__, "exit_test": W.EXIT_BRIDGE})
    nodes = orc.interface_nodes(spec.n, spec.sx, spec.sy)
    g = gpu_sums(spec)
    E = orc.bmap_tables(spec.n, spec.bmap_mode, spec.family, spec.coef_mode, spec.params)
    o = orc.mc_nodes(spec.n, nodes, E, spec.family, spec.coef_mode, spec.params, seed=spec.seed,
                     paths=spec.paths, dt=spec.dt, max_steps=spec.cap(), tie_delta=spec.tie(),
                     exit_test=1)
    _compare_fp64(orc, spec, g, o, nodes)
    # the bridge ends paths earlier than the end-of-step test
    g0 = gpu_sums(W.small_parity_cases()[case])
    assert g["steps"].sum() < g0["steps"].sum()


def test_fp32_bridge_paired_with_fp64(orc):
    spec = W.MeshSpec(**{**W.small_parity_cases()[1].__dict__, "exit_test": W.EXIT_BRIDGE})
    nodes = orc.interface_nodes(spec.n, spec.sx, spec.sy)
    g64 = gpu_sums(spec, precision=W.FP64)
    g32 = gpu_sums(spec, precision=W.FP32_STEP)
    m64, se64 = gpu_means(g64, spec.n, nodes)
    m32, _ = gpu_means(g32, spec.n, nodes)
    assert np.all(np.abs(m32 - m64) <= se64)
    assert abs(int(g32["steps"].sum()) - int(g64["steps"].sum())) / g64["steps"].sum() < 2e-3


@pytest.mark.parametrize("precision", [W.FP64, W.FP32_STEP])
def test_outputs_stay_inside_their_buffers(precision):
    """Canary rows after every device output (means, std-errs, node sums,
    mesh, smoothed mesh) are untouched: no kernel writes past its rows."""
    import torch
    from paper_1310_3435_gb300 import native as N
    spec = W.small_parity_cases()[1]
    pad = 7
    with gpu_plan(spec) as P:
        m = P.n_nodes
        mean = torch.full((m + pad, 2), float("nan"), dtype=torch.float64, device="cuda")
        se = torch.full((m + pad, 2), float("nan"), dtype=torch.float64, device="cuda")
        N.sdd_interface_mc(P.handle, P.mc_params(precision=precision), mean[:m], se[:m])
        sums = torch.full((m + pad, 12), -7, dtype=torch.int64, device="cuda")
        N.sdd_interface_mc_sums(P.handle, P.mc_params(precision=precision), sums[:m])
        n = spec.n
        mesh = torch.full((n * n * 2 + pad,), float("nan"), dtype=torch.float64, device="cuda")
        N.sdd_subdomain_solve(P.handle, mean[:m], P.solve_params(), mesh[:n * n * 2])
        N.sdd_mesh_smooth(P.handle, mesh[:n * n * 2], 3, 0.2 / (n - 1) ** 2, 1.0)
        torch.cuda.synchronize()
        assert torch.isfinite(mean[:m]).all() and torch.isfinite(se[:m]).all()
        assert torch.isnan(mean[m:]).all() and torch.isnan(se[m:]).all()
        assert (sums[m:] == -7).all()
        assert torch.isfinite(mesh[:n * n * 2]).all() and torch.isnan(mesh[n * n * 2:]).all()


def test_ring_workload_at_full_size_matches_the_oracle_on_sampled_nodes(orc):
    """The bench workload as the bench times it (257 x 257, 4 x 4, ring,
    N = 1e5, dt = 1e-5, FP32 stepping, one single-mesh launch): two sampled
    nodes, one on the ring's steep flank and one inside it, against the FP64
    oracle on the same 1e5 Philox streams (run in path ranges over the host
    cores).  The paired difference is the precision bias: within half a
    standard error, and the step counts within 1e-3."""
    from concurrent.futures import ThreadPoolExecutor
    from paper_1310_3435_gb300 import native as N
    spec = W.config2()
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
                            tie_delta=spec.tie(), node_ids=[k], threads=1, path_begin=q * per)

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
        assert abs(int(g["steps"][k]) - steps) / steps < 1e-3


def test_largest_grid_and_table(orc):
    """The largest grid a plan takes (n = 16385, 2 x 2: 32765 interface nodes,
    interface lines 8192 apart from the sides) with a few paths per node, and
    the largest density table (4097 x 4097): counts and sampled nodes against
    the oracle in FP64, and FP32 paired with FP64."""
    from paper_1310_3435_gb300 import native as N
    spec = W.MeshSpec(n=16385, sx=2, sy=2, family=W.FAMILY_RING,
                      params=(10.0, 0.5, 0.5, 50.0, 0.25), paths=8, dt=1e-4, seed=2)
    with gpu_plan(spec) as P:
        assert P.n_nodes == 2 * 16383 - 1
        g = N.sdd_interface_mc_sums(P.handle, P.mc_params())
        g32 = N.sdd_interface_mc_sums(P.handle, P.mc_params(precision=W.FP32_STEP))
        nodes = P.nodes()
    assert np.all(g["paths"] == 8) and np.all(g32["paths"] == 8)
    pick = np.linspace(0, len(nodes) - 1, 12).astype(int)
    o = oracle_sums(orc, spec, nodes=nodes[pick], node_ids=pick)
    _compare_fp64(orc, spec, g[pick], o, nodes[pick])
    m64, se64 = gpu_means(g, spec.n, nodes)
    m32, _ = gpu_means(g32, spec.n, nodes)
    assert np.mean(np.abs(m32 - m64)) < 0.1 * np.mean(se64)

    tn = 4097
    table = W.table_params(W.smooth_field(tn, seed=5, amplitude=1.0, modes=3))
    spec = W.MeshSpec(n=129, sx=2, sy=2, family=W.FAMILY_TABLE, params=table, paths=256,
                      dt=1e-4, seed=3)
    nodes = orc.interface_nodes(spec.n, spec.sx, spec.sy)
    pick = np.arange(0, len(nodes), 25)
    g = gpu_sums(spec)
    o = oracle_sums(orc, spec, nodes=nodes[pick], node_ids=pick)
    _compare_fp64(orc, spec, g[pick], o, nodes[pick])

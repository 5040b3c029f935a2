"""The tabulated density (a table of ln w, bilinear) on the GPU against the
oracle: FP64 Monte Carlo parity, FP32 paired with FP64, mesh generation,
quality and placement, batches, and argument checks."""
from dataclasses import replace

import numpy as np
import pytest

import workloads as W
from gpu_helpers import gpu_means, gpu_plan, gpu_sums

pytestmark = pytest.mark.gpu

REL_FP64 = 1e-12


def _spec(tn=17, seed=2, **kw):
    p = W.table_params(W.smooth_field(tn, seed=seed, amplitude=1.2))
    base = dict(n=21, sx=3, sy=2, family=W.FAMILY_TABLE, params=p, paths=700, dt=1e-4,
                seed=4, coef_mode=W.COEF_W, label="table %d" % tn)
    base.update(kw)
    return W.MeshSpec(**base)


def _oracle(orc, spec, nodes):
    E = orc.bmap_tables(spec.n, spec.bmap_mode, spec.family, spec.coef_mode, spec.params)
    return orc.mc_nodes(spec.n, nodes, E, spec.family, spec.coef_mode, spec.params,
                        seed=spec.seed, paths=spec.paths, dt=spec.dt, max_steps=spec.cap(),
                        tie_delta=spec.tie(), exit_test=spec.exit_test, stepper=spec.stepper)


@pytest.mark.parametrize("variant", ["plain", "inv_w_paper1d", "bridge", "exponential"])
def test_fp64_table_matches_oracle(orc, variant):
    spec = {"plain": _spec(),
            "inv_w_paper1d": _spec(coef_mode=W.COEF_INV_W, bmap_mode=W.BMAP_PAPER_1D, tn=9),
            "bridge": _spec(exit_test=W.EXIT_BRIDGE, tn=33),
            "exponential": _spec(stepper=W.STEP_EXPONENTIAL, exit_test=W.EXIT_BRIDGE)}[variant]
    nodes = orc.interface_nodes(spec.n, spec.sx, spec.sy)
    g = gpu_sums(spec)
    o = _oracle(orc, spec, nodes)
    assert np.array_equal(g["paths"], o["paths"])
    clean = (g["ties"] == 0) & (o["ties"] == 0)
    assert np.array_equal(g["steps"][clean], o["steps"][clean])
    mg, _ = gpu_means(g, spec.n, nodes, nt=True)
    mo, _ = orc.mc_estimate(nodes, spec.n, o["S_nt"], o["Q_nt"], o["paths"] - o["ties"])
    tol = 1e-11 if spec.stepper == W.STEP_EXPONENTIAL else REL_FP64
    assert np.max(np.abs(mg - mo) / np.abs(mo)) <= tol


def test_fp32_table_paired_with_fp64(orc):
    spec = _spec(paths=1500)
    nodes = orc.interface_nodes(spec.n, spec.sx, spec.sy)
    g64 = gpu_sums(spec, precision=W.FP64)
    g32 = gpu_sums(spec, precision=W.FP32_STEP)
    m64, se64 = gpu_means(g64, spec.n, nodes)
    m32, _ = gpu_means(g32, spec.n, nodes)
    d = np.abs(m32 - m64)
    assert np.all(d <= 0.5 * se64) and d.max() < 1e-3
    assert abs((m32 - m64).mean()) < 0.1 * se64.mean()


@pytest.mark.parametrize("solver", [W.SOLVER_SOR, W.SOLVER_CG_FP32_REFINE])
def test_table_mesh_generation_matches_oracle(orc, solver):
    from paper_1310_3435_gb300 import native as N
    spec = _spec(solver=solver, tol=1e-13, bmap_mode=W.BMAP_PAPER_1D)
    nodes = orc.interface_nodes(spec.n, spec.sx, spec.sy)
    o = _oracle(orc, spec, nodes)
    mo, _ = orc.mc_estimate(nodes, spec.n, o["S_all"], o["Q_all"], o["paths"])
    E = orc.bmap_tables(spec.n, spec.bmap_mode, spec.family, spec.coef_mode, spec.params)
    ref = orc.stitch(spec.n, spec.sx, spec.sy, E, mo, spec.family, spec.coef_mode, spec.params)
    with gpu_plan(spec) as P:
        assert np.allclose(np.asarray(P.edges()).ravel(), E.ravel(), rtol=0, atol=1e-13)
        mesh = np.zeros((spec.n, spec.n, 2))
        ms, ss = N.sdd_mesh_generate(P.handle, P.mc_params(), P.solve_params(), mesh)
        assert ss.converged == ss.subdomains
        q = N.sdd_mesh_quality(P.handle, mesh, ref)
    assert np.max(np.abs(mesh - ref)) < 1e-10
    want = orc.mesh_quality(mesh, ref, spec.family, spec.coef_mode, spec.params)
    assert q["l_inf"] == pytest.approx(want["l_inf"], rel=1e-12, abs=1e-15)
    assert q["q_max"] == pytest.approx(want["q_max"], rel=1e-12)


def test_table_extrema_placement_matches_oracle(orc):
    from paper_1310_3435_gb300 import native as N
    spec = _spec(n=65, sx=2, sy=2, tn=9)
    want = orc.placement(spec.n, spec.sx, spec.sy, 2, family=spec.family, params=spec.params)
    with gpu_plan(spec) as P:
        N.sdd_plan_set_placement(P.handle, N.SDD_PLACE_EXTREMA, 0)
        mask, n_mc = N.sdd_plan_placement(P.handle)
    assert np.array_equal(mask.astype(bool), want) and n_mc == int(want.sum())


def test_batch_with_tables_equals_single_runs():
    from paper_1310_3435_gb300 import native as N
    specs = [_spec(precision=W.FP32_STEP), _spec(tn=5, seed=7, precision=W.FP32_STEP),
             replace(W.small_parity_cases()[1], precision=W.FP32_STEP), _spec()]
    plans = [gpu_plan(s) for s in specs]
    try:
        alone = []
        for P in plans:
            N.sdd_interface_mc(P.handle, P.mc_params())
            m = np.zeros((P.n_nodes, 2))
            N.sdd_plan_results(P.handle, None, m, None)
            alone.append(m)
        with N.Batch(plans) as B:
            B.run()
            for k, P in enumerate(plans):
                B.stats(k)
                m = np.zeros((P.n_nodes, 2))
                N.sdd_plan_results(P.handle, None, m, None)
                assert np.array_equal(m, alone[k]), k
    finally:
        for P in plans:
            P.close()


def test_table_arguments_are_checked():
    from paper_1310_3435_gb300 import native as N
    bad = np.zeros((4, 4))
    bad[1, 2] = np.nan
    for params in (W.table_params(bad), (1.0, 0.0)):
        with pytest.raises(N.SddError):
            N.sdd_mesh_plan(9, 2, 2, N.make_density(W.FAMILY_TABLE, params))
    # the allocation-free entry point takes analytic families only
    import torch
    spec = _spec()
    with gpu_plan(spec) as P:
        nodes = torch.from_numpy(P.nodes().astype(np.int32)).cuda()
        edges = torch.from_numpy(P.edges()).cuda()
        mean = torch.zeros((P.n_nodes, 2), dtype=torch.float64, device="cuda")
        with pytest.raises(N.SddError):
            N.sdd_interface_mc_static(spec.n, nodes, edges, P.density, P.mc_params(), mean)

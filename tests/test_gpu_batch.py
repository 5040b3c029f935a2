"""Batched generation of uneven meshes (one path launch per density class,
one solve launch for every subdomain), with and without CUDA-graph replay:
every mesh's results are bitwise the same as when it runs alone."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import gpu_plan

pytestmark = pytest.mark.gpu


def _mix():
    specs = W.config3(count=5, seed=3, paths=640, dt=2e-4)
    specs += [
        W.config1(paths=512, precision=W.FP64),
        W.MeshSpec(n=41, sx=3, sy=2, family=W.FAMILY_RING, params=(10.0, 0.5, 0.5, 50.0, 0.25),
                   paths=700, dt=1e-4, seed=9, precision=W.FP32_STEP,
                   solver=W.SOLVER_CG_FP32_REFINE),
        W.MeshSpec(n=37, sx=2, sy=4, family=W.FAMILY_RIDGE, params=(20.0, 200.0, 0.3, 0.2, 1.0),
                   paths=333, dt=1e-4, seed=4, precision=W.FP32_STEP, coef_mode=W.COEF_INV_W),
        W.MeshSpec(n=29, sx=2, sy=2, family=W.FAMILY_BUMPS,
                   params=W.bumps((8.0, 0.3, 0.6, 30.0, 10.0), (3.0, 0.7, 0.2, 80.0, 80.0),
                                  (2.0, 0.5, 0.5, 20.0, 20.0), (1.0, 0.2, 0.8, 40.0, 40.0)),
                   paths=400, dt=1e-4, seed=5, precision=W.FP32_STEP),
    ]
    return specs


def _alone(spec):
    from paper_1310_3435_gb300 import native as N
    with gpu_plan(spec) as P:
        mesh = np.zeros((spec.n, spec.n, 2))
        mean = np.zeros((P.n_nodes, 2))
        se = np.zeros((P.n_nodes, 2))
        ms, ss = N.sdd_mesh_generate(P.handle, P.mc_params(), P.solve_params(), mesh, mean, se)
        return mesh, mean, se, ms


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_alone(use_graph):
    import torch
    from paper_1310_3435_gb300 import native as N
    specs = _mix()
    alone = [_alone(s) for s in specs]
    plans = [gpu_plan(s) for s in specs]
    stream = torch.cuda.Stream()
    with N.Batch(plans) as B:
        for rep in range(2):                       # second run replays the graph
            B.run(use_graph=use_graph, stream=stream)
            stream.synchronize()
            for i, (spec, P) in enumerate(zip(specs, plans)):
                mesh = np.zeros((spec.n, spec.n, 2))
                mean = np.zeros((P.n_nodes, 2))
                se = np.zeros((P.n_nodes, 2))
                N.sdd_plan_results(P.handle, mesh, mean, se)
                am, amean, ase, ams = alone[i]
                assert np.array_equal(mean, amean), (i, spec.label)
                assert np.array_equal(se, ase), (i, spec.label)
                assert np.array_equal(mesh, am), (i, spec.label)
                ms, ss = B.stats(i)
                assert ms.path_steps == ams.path_steps and ms.paths == ams.paths
                assert ss.converged == ss.subdomains
    for P in plans:
        P.close()


def test_batch_launch_count_and_validation():
    from paper_1310_3435_gb300 import native as N
    import torch
    specs = W.config3(count=4, seed=1, paths=256, dt=2e-4)
    plans = [gpu_plan(s) for s in specs]
    with N.Batch(plans) as B:
        stream = torch.cuda.Stream()
        before = N.sdd_kernel_launches()
        B.run(stream=stream)
        stream.synchronize()
        # first run: the four plans' edge coefficients, then the run itself
        assert N.sdd_kernel_launches() - before == 4 + 5
        before = N.sdd_kernel_launches()
        B.run(stream=stream)
        stream.synchronize()
        # one density class (one bump, FP32): path + reduce, fill, coons + solve
        assert N.sdd_kernel_launches() - before == 5
    with pytest.raises(N.SddError):
        N.sdd_batch_create([plans[0].handle, plans[0].handle], [plans[0].mc_params()] * 2,
                           [plans[0].solve_params()] * 2)
    with pytest.raises(N.SddError):
        with N.Batch(plans[:1]) as B:
            B.run(use_graph=True, stream=None)     # graphs need a non-default stream
    for P in plans:
        P.close()


def test_autotuned_parameters_are_valid_and_keep_results(tmp_path):
    import torch
    from paper_1310_3435_gb300 import autotune
    from paper_1310_3435_gb300 import native as N
    spec = W.config3(count=1, seed=4, paths=512, dt=2e-4)[0]
    tuner = autotune.Autotuner(path=str(tmp_path / "t.json"), probe_paths=256)
    pick = tuner.tune(spec)
    assert pick["chunk"] == 0 and pick["block_threads"] in autotune.SOLVE_THREADS
    assert tuner.timed == 3                                       # FP32: solve only
    assert tuner.tune(spec) == pick and tuner.timed == 3          # cached
    base = _alone(spec)
    with gpu_plan(spec) as P:
        mesh = np.zeros((spec.n, spec.n, 2))
        mean = np.zeros((P.n_nodes, 2))
        se = np.zeros((P.n_nodes, 2))
        N.sdd_mesh_generate(P.handle, P.mc_params(chunk=pick["chunk"]),
                            P.solve_params(block_threads=pick["block_threads"]), mesh, mean, se)
    assert np.allclose(mean, base[1], rtol=0, atol=1e-14)
    # CG dot products are reduced over the CTA's threads: meshes agree to the
    # solve tolerance (relative residual 1e-10), not bit for bit
    assert np.max(np.abs(mesh - base[0])) < 1e-8, np.max(np.abs(mesh - base[0]))


def test_uneven_batch_at_full_size_matches_the_oracle_on_sampled_nodes(orc):
    """The batched workload as the bench times it (256 uneven meshes,
    n in {65, 129, 257, 513}, splits 2..8, one bump each, N = 2e4 paths,
    dt = 5e-5, FP32 stepping, one batch replayed as a CUDA graph; the bench's
    autotuned chunk sizes leave the sums unchanged, they are exact): every
    mesh's counts and solves, and two nodes of each of six meshes (one of
    each grid size among them; one node next to the bump, one drawn at
    random) against the FP64 oracle on the same 2e4 Philox streams.  The
    paired difference is the precision bias: within half a standard error."""
    from concurrent.futures import ThreadPoolExecutor
    import torch
    from paper_1310_3435_gb300 import native as N
    specs = W.config3()
    assert len(specs) == 256 and {s.n for s in specs} == {65, 129, 257, 513}
    plans = [gpu_plan(s) for s in specs]
    means = []
    try:
        stream = torch.cuda.Stream()
        with N.Batch(plans) as B:
            B.run(use_graph=True, stream=stream)
            stream.synchronize()
            for i, (spec, P) in enumerate(zip(specs, plans)):
                ms, ss = B.stats(i)
                # every path scored; paths still inside at the step cap (2 / dt
                # steps, scored at the nearest side) stay rare
                assert ms.paths == spec.paths * P.n_nodes and ms.non_exits <= 1e-3 * ms.paths, i
                assert ss.converged == ss.subdomains, i
                mean = np.zeros((P.n_nodes, 2))
                se = np.zeros((P.n_nodes, 2))
                N.sdd_plan_results(P.handle, None, mean, se)
                assert np.all(np.isfinite(mean)) and np.all((mean > 0) & (mean < 1)), i
                means.append((mean, se, P.nodes()))
    finally:
        for P in plans:
            P.close()

    rng = np.random.default_rng(11)
    picked = []
    for n in (65, 129, 257, 513):
        picked.append(next(i for i, s in enumerate(specs) if s.n == n))
    picked += [int(i) for i in rng.choice([i for i in range(256) if i not in picked], 2,
                                          replace=False)]
    parts = 4
    jobs = []
    for i in picked:
        spec = specs[i]
        nodes = means[i][2]
        cs, ct = spec.params[2], spec.params[3]     # bumps: (count, A, cs, ct, ks, kt)
        near = int(np.argmin(np.hypot(nodes[:, 0] / (spec.n - 1.0) - cs,
                                      nodes[:, 1] / (spec.n - 1.0) - ct)))
        for k in (near, int(rng.integers(len(nodes)))):
            jobs += [(i, k, q) for q in range(parts)]
    edges = {i: orc.bmap_tables(specs[i].n, specs[i].bmap_mode, specs[i].family,
                                specs[i].coef_mode, specs[i].params) for i in picked}

    def run(job):
        i, k, q = job
        spec = specs[i]
        per = spec.paths // parts
        return orc.mc_nodes(spec.n, means[i][2][[k]], edges[i], spec.family, spec.coef_mode,
                            spec.params, seed=spec.seed, paths=per, dt=spec.dt,
                            max_steps=spec.cap(), tie_delta=spec.tie(), node_ids=[k],
                            threads=1, path_begin=q * per)

    with ThreadPoolExecutor(max_workers=orc.default_threads()) as ex:
        outs = list(ex.map(run, jobs))
    for a in range(0, len(jobs), parts):
        i, k, _ = jobs[a]
        spec = specs[i]
        mine = outs[a:a + parts]
        S = sum(o["S_all"][0] for o in mine)
        Q = sum(o["Q_all"][0] for o in mine)
        nodes = means[i][2][[k]]
        mo, so = orc.mc_estimate(nodes, spec.n, S[None, :], Q[None, :], [spec.paths])
        mg = means[i][0][[k]]
        assert np.all(np.abs(mg - mo) <= 0.5 * so), (spec.label, k, mg, mo, so)

"""Continuous-batching server: requests arriving while others run are
admitted, batched and overlapped on the device, and every result is bitwise
the same as the same request run alone: one run of all its paths, the
pilot's included (the server's final run continues the pilot's)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _alone(spec, paths, chunk):
    """One run of all `paths` paths (the work-item size the server used)."""
    from paper_1310_3435_gb300 import native as N
    with N.Plan(spec) as P:
        mesh = np.zeros((spec.n, spec.n, 2))
        mean = np.zeros((P.n_nodes, 2))
        se = np.zeros((P.n_nodes, 2))
        N.sdd_mesh_generate(P.handle, P.mc_params(paths=paths, chunk=chunk), P.solve_params(),
                            mesh, mean, se, allow_not_converged=True)
        return mesh, mean, se


def test_served_results_equal_alone():
    from paper_1310_3435_gb300 import serving as S
    arrivals = W.config5(count=14, rate=400.0, seed=7, n_max=129)
    reqs = [S.Request(i, a.spec, a.t) for i, a in enumerate(arrivals)]
    srv = S.Server(hbm_budget=2e9, n_streams=2, max_batch=4, target_stderr=4e-3,
                   pilot_paths=512, min_paths=512)
    res = srv.run(reqs)
    assert sorted(r.rid for r in res) == list(range(len(reqs)))
    assert srv.launches >= 3                         # several batches, some overlapping
    for r in res:
        assert r.max_stderr <= 4e-3 * 1.25           # pilot-chosen N meets the target
        mesh, mean, se = _alone(r.spec, r.paths, srv.chunk)    # pilot paths included
        assert np.array_equal(r.mean, mean), r.rid
        assert np.array_equal(r.stderr, se), r.rid
        assert np.array_equal(r.mesh, mesh), r.rid
    summ = S.summarize(res)
    assert summ["requests"] == len(reqs) and summ["p50_s"] <= summ["p99_s"]
    assert srv.used == 0


def test_admission_respects_the_memory_budget():
    from paper_1310_3435_gb300 import serving as S
    arrivals = W.config5(count=6, rate=1000.0, seed=2, n_max=97)
    reqs = [S.Request(i, a.spec, a.t) for i, a in enumerate(arrivals)]
    one = max(S.device_bytes(a.spec.n, a.spec.n_interface_nodes(), 2048) for a in arrivals)
    srv = S.Server(hbm_budget=1.5 * one, n_streams=2, max_batch=8, target_stderr=None)
    res = srv.run([S.Request(r.rid, W.MeshSpec(**{**r.spec.__dict__, "paths": 2048}), r.arrival)
                   for r in reqs])
    assert len(res) == len(reqs)
    assert srv.peak_used <= 1.5 * one + 1

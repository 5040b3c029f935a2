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


def _auto_chunk_raised(paths, n_nodes, sms, max_items=55185):
    """The work-item size the allocation-free entry point picks for chunk = 0:
    the library's automatic size, doubled (up to 8192) until the items fit."""
    from paper_1310_3435_gb300 import serving as S
    c = S.auto_chunk_host(paths, n_nodes, sms)
    while n_nodes * -(-paths // c) > max_items and c < 8192:
        c *= 2
    return c


def test_static_scratch_raises_the_automatic_chunk_until_the_items_fit():
    """7105 nodes x N = 1000 need more work items at the automatic size than
    the array holds, so the call raises the size; its estimates equal the
    plan entry point's at that size, and its statistics are the plan run's."""
    import torch
    from paper_1310_3435_gb300 import native as N
    spec = W.MeshSpec(n=513, sx=8, sy=8, family=W.FAMILY_BUMPS,
                      params=W.bumps((10.0, 0.4, 0.6, 60.0, 60.0)), paths=1000, dt=5e-5,
                      seed=3, precision=W.FP32_STEP, max_steps=64)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    with N.Plan(spec) as P:
        assert P.n_nodes == 7105
        chunk = _auto_chunk_raised(spec.paths, P.n_nodes, sms)
        from paper_1310_3435_gb300 import serving as S
        assert P.n_nodes * -(-spec.paths // S.auto_chunk_host(spec.paths, P.n_nodes, sms)) > 55185
        mean_ref = np.zeros((P.n_nodes, 2))
        se_ref = np.zeros((P.n_nodes, 2))
        st_ref = N.sdd_interface_mc(P.handle, P.mc_params(chunk=chunk), mean_ref, se_ref)
        nodes = torch.from_numpy(P.nodes()).cuda()
        edges = torch.from_numpy(np.ascontiguousarray(P.edges())).cuda()
        dens = P.density
    stream = torch.cuda.Stream()
    mean = torch.zeros((nodes.shape[0], 2), dtype=torch.float64, device="cuda")
    se = torch.zeros_like(mean)
    mc = N.mc_params(spec.paths, spec.dt, spec.seed, spec.precision, chunk=0,
                     max_steps=spec.max_steps)
    N.sdd_interface_mc_static(spec.n, nodes, edges, dens, mc, mean, se, stream=stream)
    st = N.sdd_interface_mc_static_stats(stream)
    assert np.allclose(mean.cpu().numpy(), mean_ref, rtol=1e-12, atol=0)
    assert np.allclose(se.cpu().numpy(), se_ref, rtol=1e-12, atol=0)
    assert (st.paths, st.path_steps, st.ties, st.non_exits) == (
        st_ref.paths, st_ref.path_steps, st_ref.ties, st_ref.non_exits)
    # the size the call picked is the one computed here: an explicit call at
    # that size gives bitwise the same estimates
    mean2 = torch.zeros_like(mean)
    N.sdd_interface_mc_static(spec.n, nodes, edges, dens,
                              N.mc_params(spec.paths, spec.dt, spec.seed, spec.precision,
                                          chunk=chunk, max_steps=spec.max_steps), mean2,
                              stream=stream)
    stream.synchronize()
    assert torch.equal(mean, mean2)


def test_static_scratch_refuses_short_or_misaligned_buffers_without_launching():
    import torch
    from paper_1310_3435_gb300 import native as N
    spec = W.config1(paths=256)
    with N.Plan(spec) as P:
        nodes = torch.from_numpy(P.nodes()).cuda()
        edges = torch.from_numpy(np.ascontiguousarray(P.edges())).cuda().reshape(-1)
        dens = P.density
    m = nodes.shape[0]
    mean = torch.zeros((m, 2), dtype=torch.float64, device="cuda")
    mc = N.mc_params(spec.paths, spec.dt, spec.seed, spec.precision)
    # a buffer at the very end of its own allocation (a 256 MiB tensor is one
    # allocation of exactly that size), one element too short for the tables
    torch.cuda.empty_cache()
    big = torch.zeros(2 ** 25, dtype=torch.float64, device="cuda")
    short = big[-(8 * spec.n - 1):]
    short.copy_(edges[:8 * spec.n - 1])
    twice = torch.zeros(2 * m + 1, dtype=torch.int32, device="cuda")
    twice[1:].copy_(nodes.reshape(-1))
    odd = twice[1:].reshape(m, 2)                    # 4 bytes past an 8-byte boundary
    before = N.sdd_kernel_launches()
    for args, what in (((short, mean, nodes), "edges needs"),
                       ((edges, mean, odd), "nodes must be aligned")):
        e_, mean_, nodes_ = args
        with pytest.raises(N.SddError) as e:
            N.sdd_interface_mc_static(spec.n, nodes_, e_, dens, mc, mean_)
        assert e.value.code == N.SDD_ERR_INVALID_ARG
        assert what in N.sdd_last_error(), N.sdd_last_error()
    with pytest.raises(N.SddError) as e:             # host memory is not taken
        N.sdd_interface_mc_static(spec.n, nodes, edges.cpu(), dens, mc, mean)
    assert "device memory" in N.sdd_last_error()
    assert N.sdd_kernel_launches() == before
    del big


"""Host logic of the continuous-batching server, on the CPU: admission by
memory budget, pilot-chosen paths, batching on a bounded number of streams,
overlap of batches, completion order.  The library and CUDA streams/events are
replaced by stand-ins whose "kernels" finish after a set wall-clock time."""
import math
import time
import types

import pytest

import workloads as W
from paper_1310_3435_gb300 import serving as S


class FakeEvent:
    def __init__(self):
        self.t = None

    def record(self, stream):
        self.t = stream.busy_until

    def query(self):
        return time.perf_counter() >= self.t


class FakeStream:
    def __init__(self):
        self.busy_until = time.perf_counter()

    def enqueue(self, seconds):
        self.busy_until = max(self.busy_until, time.perf_counter()) + seconds

    def synchronize(self):
        while time.perf_counter() < self.busy_until:
            time.sleep(1e-4)


class FakeCuda:
    Stream = FakeStream
    Event = FakeEvent

    @staticmethod
    def current_device():
        return 0

    @staticmethod
    def get_device_properties(dev):
        return types.SimpleNamespace(multi_processor_count=152)


class FakeLib:
    """Plans know their node count; a pilot reports std-err sigma/sqrt(N);
    a batch takes 2 ms per mesh."""
    SIGMA = 0.05

    def __init__(self):
        self.live_plans = 0
        self.max_live = 0
        self.batches = []
        self.concurrent = 0
        self.max_concurrent = 0
        self.final_mcs = []

    class _Plan:
        def __init__(self, lib, spec):
            self.lib, self.spec, self.n = lib, spec, spec.n
            self.n_nodes = spec.n_interface_nodes()
            self.handle = self
            lib.live_plans += 1
            lib.max_live = max(lib.max_live, lib.live_plans)
            self.pilot_paths = None

        def mc_params(self, **kw):
            return dict(paths=kw.get("paths", self.spec.paths), chunk=kw.get("chunk", 0),
                        path_begin=kw.get("path_begin", 0))

        def solve_params(self):
            return {}

        def close(self):
            if self.handle is not None:
                self.lib.live_plans -= 1
                self.handle = None

    def Plan(self, spec):
        return FakeLib._Plan(self, spec)

    def sdd_interface_mc(self, handle, mc, want_stats=False, stream=None):
        handle.pilot_paths = mc["paths"]
        handle.pilot_chunk = mc["chunk"]
        stream.enqueue(0.001)

    def sdd_plan_last_mc_stats(self, handle):
        return types.SimpleNamespace(max_stderr=self.SIGMA / math.sqrt(handle.pilot_paths))

    class _Batch:
        def __init__(self, lib, plans, mcs, sps):
            self.lib, self.plans, self.mcs = lib, plans, mcs
            lib.batches.append([m["paths"] for m in mcs])
            lib.final_mcs.extend((p, m) for p, m in zip(plans, mcs))

        def run(self, use_graph=False, stream=None):
            stream.enqueue(0.002 * len(self.plans))
            self.stream = stream

        def stats(self, k, allow_not_converged=False):
            paths = self.mcs[k]["paths"]
            return (types.SimpleNamespace(path_steps=1000 * paths,
                                          max_stderr=FakeLib.SIGMA / math.sqrt(paths)), None)

        def close(self):
            pass

    def Batch(self, plans, mcs, sps):
        return FakeLib._Batch(self, plans, mcs, sps)

    def sdd_plan_results(self, handle, mesh, mean, se, stream=None):
        mesh[...] = 0.0
        mean[...] = 0.0
        se[...] = 0.0


def _requests(count, rate, seed=1):
    arr = W.config5(count=count, rate=rate, seed=seed, n_max=65)
    return [S.Request(i, a.spec, a.t) for i, a in enumerate(arr)]


def test_every_request_served_with_pilot_paths():
    lib = FakeLib()
    srv = S.Server(hbm_budget=1e12, n_streams=3, max_batch=8, target_stderr=1e-3,
                   pilot_paths=1024, backend=lib, cuda=FakeCuda, sms=152)
    res = srv.run(_requests(40, rate=2000.0))
    assert sorted(r.rid for r in res) == list(range(40))
    want = math.ceil((FakeLib.SIGMA / 1e-3) ** 2)           # 2500 paths
    assert all(r.paths == want for r in res)
    assert all(r.max_stderr <= 1e-3 for r in res)
    assert srv.used == 0 and lib.live_plans == 0
    assert all(len(b) <= 8 for b in lib.batches)
    assert len(lib.batches) >= 5                        # requests batched as they came
    s = S.summarize(res)
    assert s["p50_s"] <= s["p99_s"] and s["requests"] == 40


def test_admission_waits_for_memory():
    lib = FakeLib()
    reqs = _requests(12, rate=5000.0)
    one = max(S.device_bytes(r.spec.n, r.spec.n_interface_nodes(), r.spec.paths) for r in reqs)
    srv = S.Server(hbm_budget=2.2 * one, n_streams=3, max_batch=8, target_stderr=None,
                   backend=lib, cuda=FakeCuda, sms=152)
    res = srv.run(reqs)
    assert len(res) == 12
    assert srv.peak_used <= 2.2 * one                 # never more than the budget allows
    assert lib.max_live < 12                          # admission had to wait


def test_batches_overlap_on_streams_and_latency_includes_queueing():
    lib = FakeLib()
    reqs = _requests(30, rate=10000.0)
    srv = S.Server(hbm_budget=1e12, n_streams=2, max_batch=3, target_stderr=None,
                   backend=lib, cuda=FakeCuda, sms=152)
    res = srv.run(reqs)
    starts = sorted((r.started, r.done) for r in res)
    # with two streams, some batch starts before an earlier one is done
    assert any(b[0] < a[1] for a, b in zip(starts, starts[1:]) if b[0] > a[0])
    assert all(r.done >= r.started >= r.arrival for r in res)


class FaultyLib(FakeLib):
    """Failures injected on the host: the plan of request `bad_plan` cannot be
    built (a malformed or oversized request), and every batch holding request
    `bad_batch` fails to launch."""

    def __init__(self, bad_plan, bad_batch):
        super().__init__()
        self.bad_plan, self.bad_batch = bad_plan, bad_batch

    def Plan(self, spec):
        if spec.label == "req%d" % self.bad_plan:
            raise RuntimeError("injected: plan allocation failed")
        return FakeLib._Plan(self, spec)

    def Batch(self, plans, mcs, sps):
        if any(p.spec.label == "req%d" % self.bad_batch for p in plans):
            raise RuntimeError("injected: batch launch failed")
        return FakeLib._Batch(self, plans, mcs, sps)


def test_failures_are_reported_and_the_server_carries_on():
    lib = FaultyLib(bad_plan=3, bad_batch=11)
    srv = S.Server(hbm_budget=1e12, n_streams=2, max_batch=4, target_stderr=1e-3,
                   pilot_paths=1024, backend=lib, cuda=FakeCuda, sms=152)
    res = srv.run(_requests(24, rate=3000.0))
    by = {r.rid: r for r in res}
    assert sorted(by) == list(range(24))              # every request gets an answer
    assert by[3].status == "failed" and "plan allocation" in by[3].error
    failed_batch = [r for r in res if r.status == "failed" and "batch launch" in r.error]
    assert 11 in {r.rid for r in failed_batch}        # its batch mates fail with it
    ok = [r for r in res if r.status == "ok"]
    assert len(ok) == 24 - 1 - len(failed_batch) and all(r.mesh is not None for r in ok)
    assert srv.used == 0 and lib.live_plans == 0      # memory and plans given back
    s = S.summarize(res)
    assert s["requests"] == len(ok) and s["failed"] == 1 + len(failed_batch)


def test_cancelled_requests():
    lib = FakeLib()
    reqs = _requests(16, rate=4000.0)
    srv = S.Server(hbm_budget=1e12, n_streams=1, max_batch=4, target_stderr=None,
                   backend=lib, cuda=FakeCuda, sms=152)
    srv.cancel(5)                                      # cancelled before it arrives
    last = reqs[-1].rid
    orig_run = FakeLib._Batch.run

    def run_and_cancel(self, use_graph=False, stream=None):
        orig_run(self, use_graph, stream)
        if any(p.spec.label == "req%d" % last for p in self.plans):
            srv.cancel(last)                           # cancelled while its batch runs
    FakeLib._Batch.run = run_and_cancel
    try:
        res = srv.run(reqs)
    finally:
        FakeLib._Batch.run = orig_run
    by = {r.rid: r for r in res}
    assert sorted(by) == list(range(16))
    assert by[5].status == "cancelled" and by[5].mesh is None
    assert by[last].status == "cancelled" and by[last].mesh is None
    assert all(r.status == "ok" for k, r in by.items() if k not in (5, last))
    assert srv.used == 0 and lib.live_plans == 0


def test_busy_fraction_is_the_union_of_device_intervals():
    trace = [("pilot", 0, 0.0, 1.0), ("batch", 0, 0.5, 2.0, 3), ("batch", 1, 3.0, 4.0, 1)]
    assert S.busy_fraction(trace) == pytest.approx(3.0 / 4.0)
    assert S.busy_fraction([]) == 0.0
    assert S.busy_fraction(trace, span=6.0) == pytest.approx(0.5)


@pytest.mark.parametrize("reuse", [True, False])
def test_final_runs_continue_the_pilots(reuse):
    """With reuse the final run of every request continues its pilot: the
    same work-item size for both (the pilot's path count) and path_begin =
    pilot paths, so the pilot's paths count in the estimate; without it the
    final run starts at path 0."""
    lib = FakeLib()
    srv = S.Server(hbm_budget=1e12, n_streams=2, max_batch=4, target_stderr=1e-3,
                   pilot_paths=512, min_paths=256, backend=lib, cuda=FakeCuda, sms=152,
                   reuse_pilot=reuse)
    res = srv.run(_requests(10, rate=3000.0))
    assert len(res) == 10 and len(lib.final_mcs) == 10
    for plan, mc in lib.final_mcs:
        if reuse:
            assert mc["path_begin"] == 512 and mc["chunk"] == 512
            assert plan.pilot_chunk == 512 and mc["paths"] >= 512
        else:
            assert mc["path_begin"] == 0 and mc["chunk"] == 0 and plan.pilot_chunk == 0
    with pytest.raises(ValueError):
        S.Server(target_stderr=1e-3, pilot_paths=1000, backend=lib, cuda=FakeCuda, sms=152)


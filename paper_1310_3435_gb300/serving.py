"""Continuous-batching server for mesh-generation requests.

Requests (grid size, subdomain split, density, boundary map, time step, seed)
arrive over time.  The server admits them while their device memory fits an
HBM budget. Each admitted request may get a pilot Monte Carlo run that picks
its paths per node for a target standard error. Admitted requests are grouped
into batches, one C-ABI batch each (one path launch per density family, one
solve launch). Up to `n_streams` batches are in flight at once on separate
CUDA streams, so a batch formed from requests that arrived while another was
running starts as soon as SMs free up, and their work overlaps on the
device. Completed batches are polled through CUDA events. Their plans are
released stream-ordered, and the memory budget is handed back.

Every request keeps its own Philox key and work-item size, so its result is
bitwise the same alone and in any mix (see tests/test_gpu_serving.py).  The
pilot's paths are not thrown away: the estimator is a sum over paths, so the
final run continues the pilot (sdd_mc_params.path_begin) and runs only the
paths the pilot did not, with a result bitwise equal to one run of N paths
of the same work-item size.
PyTorch is used for streams, events and pinned host buffers only.

Failures stay with the requests they hit: a request whose plan or pilot
cannot be built, or every request of a batch that cannot be launched, is
answered with status "failed" and the error, its memory is given back, and
the server carries on.  `cancel(rid)` drops a request that has not reached a
batch, or discards the results of one whose batch is running.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field, replace

import numpy as np

from . import native as N

SLOT_BYTES = 152            # device bytes of one work-item slot


@dataclass
class Request:
    rid: int
    spec: object                 # attributes as workloads.MeshSpec
    arrival: float = 0.0         # seconds after the server starts


@dataclass
class Result:
    rid: int
    spec: object
    paths: int
    mesh: np.ndarray
    mean: np.ndarray
    stderr: np.ndarray
    path_steps: int
    max_stderr: float
    arrival: float
    admitted: float
    started: float
    done: float
    batch: int
    status: str = "ok"           # "ok", "failed" (error holds why) or "cancelled"
    error: str = ""

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def auto_chunk_host(paths: int, n_nodes: int, sms: int) -> int:
    """Mirror of the library's automatic work-item size (for memory estimates)."""
    target = paths * n_nodes / (32.0 * 24.0 * sms)
    c = 64
    while c < 4096 and 2 * c <= target:
        c *= 2
    return min(c, ((paths + 31) // 32) * 32)


def device_bytes(n: int, n_nodes: int, paths: int, sms: int = 152, chunk: int = 0) -> int:
    """Device memory of one request's plan: tables, work-item slots, node
    outputs, mesh, edge coefficients (FP64 + FP32), the CG workspace (44 B
    per grid node) and the multigrid levels (at most 15 floats per coarse
    node: under a third of the grid plus padding rings, bounded by 24 B per
    grid node) (chunk: the work-item size, 0 = the library's automatic one)."""
    chunk = chunk or auto_chunk_host(paths, max(n_nodes, 1), sms)
    items = n_nodes * ((paths + chunk - 1) // chunk)
    return (8 * n_nodes + 64 * n + items * SLOT_BYTES + n_nodes * (96 + 32)
            + 16 * n * n + 24 * n * (n - 1) + (44 + 24) * n * n + 4096)


@dataclass
class _InFlight:
    bid: int
    batch: object
    reqs: list
    plans: list
    paths: list
    stream: object
    event: object
    started: float
    nbytes: int


class Server:
    """Admission by memory budget, pilot-chosen paths, continuous batching.

    Request states: arrived -> admitted (plan built, pilot Monte Carlo queued
    on the pilot stream) -> ready (paths per node chosen) -> in a batch on one
    of the batch streams -> done.  The host never waits for the device: pilots
    and batches are polled through CUDA events."""

    def __init__(self, hbm_budget: float = 150e9, n_streams: int = 3, max_batch: int = 256,
                 target_stderr: float | None = 1e-3, pilot_paths: int = 1024,
                 min_paths: int = 1024, max_paths: int = 4_000_000, use_graph: bool = False,
                 max_wait: float = 0.25, backend=None, cuda=None, sms: int | None = None,
                 reuse_pilot: bool = True):
        """backend / cuda: the library binding and the stream/event provider
        (default: paper_1310_3435_gb300.native and torch.cuda); tests of the
        host logic pass stand-ins.  reuse_pilot: the final run continues the
        pilot's paths (both then use work items of pilot_paths paths, which
        must be a multiple of 32 up to 8192)."""
        self.N = backend if backend is not None else N
        if cuda is None:
            import torch
            cuda = torch.cuda
        self.cuda = cuda
        self.budget = float(hbm_budget)
        self.n_streams = n_streams
        self.max_batch = max_batch
        self.target = target_stderr
        self.pilot_paths = pilot_paths
        self.reuse_pilot = bool(reuse_pilot and target_stderr)
        if self.reuse_pilot and (pilot_paths % 32 or not 32 <= pilot_paths <= 8192):
            raise ValueError("reusing the pilot needs pilot_paths a multiple of 32 up to 8192")
        self.chunk = pilot_paths if self.reuse_pilot else 0
        self.min_paths = max(min_paths, pilot_paths) if self.reuse_pilot else min_paths
        self.max_paths = max_paths
        self.use_graph = use_graph
        self.max_wait = max_wait
        self.streams = [cuda.Stream() for _ in range(n_streams)]
        self.pilot_stream = cuda.Stream()
        self.sms = sms or cuda.get_device_properties(cuda.current_device()).multi_processor_count
        self.used = 0
        self.peak_used = 0
        self.launches = 0
        self._cancel = set()
        # timeline of the last run (seconds after its start): ("pilot", rid,
        # queued, seen done) and ("batch", id, launched, seen done, requests)
        self.trace = []

    def cancel(self, rid: int) -> None:
        """Cancels request `rid`: a request not yet in a batch is dropped at
        the next turn of the loop; one whose batch is running is reported as
        cancelled (without results) when the batch completes."""
        self._cancel.add(rid)

    @staticmethod
    def _dropped(req, status, error, t, batch=-1):
        return Result(req.rid, req.spec, 0, None, None, None, 0, math.nan, req.arrival, t, t, t,
                      batch, status=status, error=error)

    def _paths_for(self, spec, pilot_stats) -> int:
        """N = ceil((sigma_max / target)^2) with sigma = pilot stderr sqrt(N_pilot)."""
        if not self.target:
            return int(spec.paths)
        sigma = pilot_stats.max_stderr * math.sqrt(self.pilot_paths)
        need = int(math.ceil((sigma / self.target) ** 2))
        return int(min(self.max_paths, max(self.min_paths, need)))

    def run(self, requests, time_scale: float = 1.0, poll_sleep: float = 0.0002):
        """Serves `requests` in real time (arrival times in seconds, divided by
        time_scale); returns the results in completion order."""
        cuda = self.cuda
        N = self.N
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        piloting = deque()            # [req, plan, event, base_bytes, t_admit]
        ready = deque()               # [req, plan, paths, nbytes, t_admit]
        inflight: list[_InFlight] = []
        results = []
        free_streams = deque(range(self.n_streams))
        bid = 0
        t0 = time.perf_counter()
        now = lambda: (time.perf_counter() - t0) * time_scale
        self.trace = []
        while pending or piloting or ready or inflight:
            progressed = False
            t = now()
            # 1. admission (FIFO) while the request's base memory fits the budget
            while pending and pending[0].arrival <= t:
                req = pending[0]
                base = device_bytes(req.spec.n, req.spec.n_interface_nodes(),
                                    self.pilot_paths if self.target else int(req.spec.paths),
                                    self.sms, self.chunk)
                if self.used + base > self.budget and (piloting or ready or inflight):
                    break                                   # wait for memory to free up
                pending.popleft()
                progressed = True
                if req.rid in self._cancel:
                    results.append(self._dropped(req, "cancelled", "", now()))
                    continue
                try:
                    plan = N.Plan(req.spec)
                except Exception as e:                  # malformed request, no memory, ...
                    results.append(self._dropped(req, "failed", str(e), now()))
                    continue
                self.used += base
                self.peak_used = max(self.peak_used, self.used)
                ev = None
                if self.target:
                    try:
                        N.sdd_interface_mc(plan.handle,
                                           plan.mc_params(paths=self.pilot_paths, chunk=self.chunk),
                                           want_stats=False, stream=self.pilot_stream)
                    except Exception as e:
                        plan.close()
                        self.used -= base
                        results.append(self._dropped(req, "failed", str(e), now()))
                        continue
                    ev = cuda.Event()
                    ev.record(self.pilot_stream)
                piloting.append([req, plan, ev, base, now()])
            # 2. pilots done -> paths per node chosen, memory re-estimated
            while piloting and (piloting[0][2] is None or piloting[0][2].query()):
                req, plan, ev, base, ta = piloting.popleft()
                progressed = True
                self.trace.append(("pilot", req.rid, ta, now()))
                try:
                    st = N.sdd_plan_last_mc_stats(plan.handle) if ev is not None else None
                    paths = self._paths_for(req.spec, st)
                except Exception as e:
                    plan.close()
                    self.used -= base
                    results.append(self._dropped(req, "failed", str(e), now()))
                    continue
                nbytes = device_bytes(req.spec.n, plan.n_nodes, paths, self.sms, self.chunk)
                self.used += nbytes - base
                self.peak_used = max(self.peak_used, self.used)
                ready.append([req, plan, paths, nbytes, ta])
            # cancelled requests leave the queues before they reach a batch
            if self._cancel:
                for q in (piloting, ready):
                    keep = deque()
                    for x in q:
                        if x[0].rid in self._cancel:
                            x[1].close()
                            self.used -= x[3]
                            results.append(self._dropped(x[0], "cancelled", "", now()))
                            progressed = True
                        else:
                            keep.append(x)
                    q.clear()
                    q.extend(keep)
            # 3. launch the ready requests as one batch on a free stream: at once
            # when the device is idle; while a batch runs, let the ready queue
            # fill up (to max_batch, or until its oldest request has waited
            # max_wait seconds) so that the next batch is a large one
            fill = (not inflight or len(ready) >= self.max_batch
                    or (ready and now() - ready[0][4] >= self.max_wait))
            if ready and free_streams and fill:
                take = [ready.popleft() for _ in range(min(self.max_batch, len(ready)))]
                plans = [x[1] for x in take]
                if self.reuse_pilot:              # continue each request's pilot
                    mcs = [p.mc_params(paths=x[2], chunk=self.chunk, path_begin=self.pilot_paths)
                           for p, x in zip(plans, take)]
                else:
                    mcs = [p.mc_params(paths=x[2]) for p, x in zip(plans, take)]
                si = free_streams.popleft()
                stream = self.streams[si]
                started = now()
                batch = None
                try:
                    batch = N.Batch(plans, mcs, [p.solve_params() for p in plans])
                    batch.run(use_graph=self.use_graph, stream=stream)
                except Exception as e:                  # the whole batch fails
                    if batch is not None:
                        batch.close()
                    for x in take:
                        x[1].close()
                        self.used -= x[3]
                        results.append(self._dropped(x[0], "failed", str(e), now(), bid))
                    free_streams.append(si)
                    bid += 1
                    progressed = True
                    continue
                ev = cuda.Event()
                ev.record(stream)
                inflight.append(_InFlight(bid, batch, [x[0] for x in take], plans,
                                          [x[2] for x in take], (si, stream), ev, started,
                                          sum(x[3] for x in take)))
                for x in take:
                    x[0].admitted_at = x[4]
                bid += 1
                self.launches += 1
                progressed = True
            # 4. completion
            still = []
            for f in inflight:
                if f.event.query():
                    done = now()
                    self.trace.append(("batch", f.bid, f.started, done, len(f.reqs)))
                    for k, (req, plan) in enumerate(zip(f.reqs, f.plans)):
                        admitted = getattr(req, "admitted_at", f.started)
                        if req.rid in self._cancel:
                            results.append(Result(req.rid, req.spec, f.paths[k], None, None, None,
                                                  0, math.nan, req.arrival, admitted, f.started,
                                                  done, f.bid, status="cancelled"))
                            continue
                        n = plan.n
                        mesh = np.empty((n, n, 2))
                        mean = np.empty((plan.n_nodes, 2))
                        se = np.empty((plan.n_nodes, 2))
                        try:
                            N.sdd_plan_results(plan.handle, mesh, mean, se, stream=f.stream[1])
                            ms, _ = f.batch.stats(k, allow_not_converged=True)
                        except Exception as e:
                            results.append(Result(req.rid, req.spec, f.paths[k], None, None, None,
                                                  0, math.nan, req.arrival, admitted, f.started,
                                                  done, f.bid, status="failed", error=str(e)))
                            continue
                        results.append(Result(req.rid, req.spec, f.paths[k], mesh, mean, se,
                                              int(ms.path_steps), float(ms.max_stderr),
                                              req.arrival, admitted, f.started, done, f.bid))
                    f.batch.close()
                    for plan in f.plans:
                        plan.close()
                    self.used -= f.nbytes
                    free_streams.append(f.stream[0])
                    progressed = True
                else:
                    still.append(f)
            inflight = still
            if not progressed:
                if pending and not (piloting or ready or inflight):
                    wait = (pending[0].arrival - now()) / time_scale
                    if wait > 0:
                        time.sleep(min(wait, 0.05))
                else:
                    time.sleep(poll_sleep)
        return results


def busy_fraction(trace, span=None) -> float:
    """Share of the run during which at least one batch or pilot was on the
    device (union of their intervals in the trace, as the host saw them)."""
    iv = sorted((e[2], e[3]) for e in trace)
    if not iv:
        return 0.0
    total, cur_s, cur_e = 0.0, iv[0][0], iv[0][1]
    for a, b in iv[1:]:
        if a > cur_e:
            total += cur_e - cur_s
            cur_s, cur_e = a, b
        else:
            cur_e = max(cur_e, b)
    total += cur_e - cur_s
    span = span if span is not None else max(e[3] for e in trace) - min(e[2] for e in trace)
    return total / span if span > 0 else 0.0


def summarize(results, wall: float | None = None) -> dict:
    """p50 / p99 latency, meshes/s and path-steps/s of a served run (over the
    requests served; failed and cancelled ones are counted apart)."""
    failed = sum(1 for r in results if r.status == "failed")
    cancelled = sum(1 for r in results if r.status == "cancelled")
    results = [r for r in results if r.status == "ok"]
    if not results:
        return {"requests": 0, "failed": failed, "cancelled": cancelled}
    lat = np.array([r.latency for r in results])
    t_first = min(r.arrival for r in results)
    t_last = max(r.done for r in results)
    span = wall if wall is not None else (t_last - t_first)
    steps = sum(r.path_steps for r in results)
    return {"requests": len(results), "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
            "meshes_per_s": len(results) / span, "path_steps_per_s": steps / span,
            "span_s": span, "max_stderr": float(max(r.max_stderr for r in results)),
            "batches": len({r.batch for r in results}), "failed": failed,
            "cancelled": cancelled}

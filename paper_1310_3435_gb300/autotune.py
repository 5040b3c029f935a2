"""Autotuner for the launch parameters of the mesh generator.

Two choices are tuned, each per bucket of similar requests and cached per GPU
in a JSON file:

* paths per work item (`chunk`) of the interface Monte Carlo in FP64
  stepping, bucketed by (density family, log2 of interface nodes x paths per
  node).  FP32 stepping keeps the automatic size: its lanes stream across work
  items, and its speed does not depend on the item size (measured);
* threads per subdomain CTA of the batched solves (256, 512, 1024), bucketed
  by (solver, log2 of the largest subdomain's interior nodes), and, for a
  whole batch, the CTA size of its one solve launch (`tune_batch_solve`).

Each candidate is timed with CUDA events on the real kernels, through the C
ABI, on a reduced copy of the request: its first `probe_paths` paths per
node for the Monte Carlo, and the full subdomain solves.  The fastest
candidate wins.  The Monte Carlo estimate does not depend on the work-item
size beyond the last bits of a compensated FP64 sum (FP32-stepping sums are
exact per item).  The CG solves reduce their dot products over the CTA's
threads, so meshes from different CTA sizes agree to the solver tolerance
rather than bit for bit.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import replace

from . import build as _build

CHUNKS = (256, 1024, 4096)
SOLVE_THREADS = (256, 512, 1024)


def cache_path(device_name: str) -> str:
    safe = "".join(ch if ch.isalnum() else "_" for ch in device_name)
    return os.environ.get("SDD_AUTOTUNE_CACHE",
                          os.path.join(_build.BUILD, "autotune_%s.json" % safe))


def mc_bucket(spec, n_nodes: int) -> str:
    work = max(1, n_nodes * int(spec.paths))
    return "mc/p%d/f%d/nb%d/w%d" % (spec.precision, spec.family,
                                    int(spec.params[0]) if spec.family == 0 else 0,
                                    int(math.log2(work)))


def largest_subdomain(spec) -> int:
    def lines(n, s):
        return [0] + [(2 * k * (n - 1) + s) // (2 * s) for k in range(1, s)] + [n - 1]
    X, Y = lines(spec.n, spec.sx), lines(spec.n, spec.sy)
    return max((X[a + 1] - X[a] - 1) * (Y[b + 1] - Y[b] - 1)
               for a in range(spec.sx) for b in range(spec.sy))


def solve_bucket(spec) -> str:
    # "mg": the CG solver is multigrid-preconditioned (timings of the former
    # diagonal preconditioner do not carry over)
    return "solve/mg/s%d/m%d" % (spec.solver, int(math.log2(max(1, largest_subdomain(spec)))))


class Autotuner:
    """tune(spec) -> {"chunk": c, "block_threads": t}; results cached."""

    def __init__(self, timer=None, device_name: str | None = None, probe_paths: int = 2048,
                 path: str | None = None):
        self._timer = timer
        if device_name is None:
            import torch
            device_name = torch.cuda.get_device_name(torch.cuda.current_device())
        self.device_name = device_name
        self.path = path or cache_path(device_name)
        self.probe_paths = probe_paths
        self.cache = {}
        if os.path.exists(self.path):
            try:
                with open(self.path) as fh:
                    self.cache = json.load(fh)
            except (OSError, ValueError):
                self.cache = {}
        self.timed = 0

    def save(self) -> None:
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        tmp = self.path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as fh:
            json.dump(self.cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    # -- timing of one candidate (CUDA events on the library's kernels) -----
    def _time(self, kind: str, spec, value) -> float:
        if self._timer is not None:
            return self._timer(kind, spec, value)
        import numpy as np
        import torch
        from . import native as N
        self.timed += 1
        stream = torch.cuda.Stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        probe = replace(spec, paths=min(int(spec.paths), self.probe_paths))
        with N.Plan(probe) as P:
            if kind == "mc":
                mc = P.mc_params(chunk=value)
                N.sdd_interface_mc(P.handle, mc, want_stats=False, stream=stream)    # warm-up
                e0.record(stream)
                N.sdd_interface_mc(P.handle, mc, want_stats=False, stream=stream)
                e1.record(stream)
            else:
                iface = torch.zeros((max(P.n_nodes, 1), 2), dtype=torch.float64, device="cuda")
                nodes = torch.from_numpy(P.nodes().astype(np.float64)).cuda() / (probe.n - 1.0)
                iface[:P.n_nodes] = nodes
                mesh = torch.zeros((probe.n, probe.n, 2), dtype=torch.float64, device="cuda")
                sp = P.solve_params(block_threads=value)
                N.sdd_subdomain_solve(P.handle, iface, sp, mesh, want_stats=False, stream=stream)
                e0.record(stream)
                N.sdd_subdomain_solve(P.handle, iface, sp, mesh, want_stats=False, stream=stream)
                e1.record(stream)
            stream.synchronize()
            return e0.elapsed_time(e1)

    def _best(self, key: str, kind: str, spec, candidates):
        if key in self.cache:
            return self.cache[key]["best"]
        times = {str(c): self._time(kind, spec, c) for c in candidates}
        best = min(candidates, key=lambda c: times[str(c)])
        self.cache[key] = {"best": best, "ms": times}
        return best

    def tune_batch_solve(self, plans, mcs, sps, candidates=(512, 1024)) -> int:
        """CTA size for the solve launch of a batch: all its subdomains run in
        one launch of one CTA size, and with many subdomains several smaller
        CTAs per SM beat one large one (their barrier waits overlap), which
        single-mesh timings do not show.  Sets each plan's interface values to
        its nodes' coordinates (one solve per plan; the solve's cost does not
        depend on the values), then times the batch's fill + solve phase per
        candidate and returns the fastest; the candidates' batches are built
        and freed here."""
        if self._timer is not None:
            return min(candidates, key=lambda c: self._timer("batch", None, c))
        import numpy as np
        import torch
        from . import native as N
        from .native import solve_params as _sp
        stream = torch.cuda.Stream()
        n_max = max(p.n for p in plans)
        mesh = torch.empty((n_max * n_max * 2,), dtype=torch.float64, device="cuda")
        for p, sp in zip(plans, sps):
            iface = np.ascontiguousarray(p.nodes() / (p.n - 1.0))
            N.sdd_subdomain_solve(p.handle, iface, sp, mesh[:p.n * p.n * 2], want_stats=False,
                                  stream=stream)
        stream.synchronize()
        best, best_ms = None, None
        for c in candidates:
            sp_c = [_sp(solver=sp.solver, tol=sp.tol, max_iter=sp.max_iter, omega=sp.omega,
                        block_threads=c) for sp in sps]
            with N.Batch(plans, mcs, sp_c) as B:
                B.run_phases(2, stream=stream)                        # warm-up
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                B.run_phases(2, stream=stream)
                e1.record(stream)
                stream.synchronize()
                ms = e0.elapsed_time(e1)
            self.timed += 1
            if best_ms is None or ms < best_ms:
                best, best_ms = c, ms
        return int(best)

    def tune(self, spec, n_nodes: int | None = None) -> dict:
        if n_nodes is None:
            n_nodes = (spec.sx - 1) * (spec.n - 2) + (spec.sy - 1) * (spec.n - 2) - (
                spec.sx - 1) * (spec.sy - 1)
        chunk = 0
        if int(spec.precision) == 0:                  # FP64 stepping: item-at-a-time lanes
            chunk = self._best(mc_bucket(spec, n_nodes), "mc", spec, CHUNKS)
        threads = self._best(solve_bucket(spec), "solve", spec, SOLVE_THREADS)
        return {"chunk": int(chunk), "block_threads": int(threads)}

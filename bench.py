"""Benchmark of the GB300 SDD mesh generator.

One step = one whole mesh generation of the 257x257, 4x4-split ring workload
(1521 interface nodes, 1e5 paths per node, dt = 1e-5, FP32 stepping with FP64
accumulation, FP32 CG + FP64 refinement to 1e-10): the interface Monte Carlo
(path kernel + per-node reduction) followed by the batched subdomain solves.
Metric: SDE path-steps per second (whole job), with meshes/s beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

--impl reference times the FP64 CPU oracle (the test oracle, as it stands)
on the host cores on a bounded sample of the same workload.
Under torchrun each rank generates its own meshes (independent problems, no
data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

# Algorithmic arithmetic operations of one FP32 path-step of the ring
# density, counted per thread:
#   Philox4x32-10 / 2 steps: 10 rounds x (2 wide multiplies counted as 2,
#   2 three-input xors, 2 key additions) = 60 -> 30 per step
#   two uniforms (shift-or + add): 4;  Box-Muller pair: 9 (4 of them MUFU);
#   ring drift: 21 (3 MUFU);  Euler-Maruyama update: 4;  exit test: 6;
#   step count and cap test: 2
OPS_PER_STEP_RING_FP32 = 30 + 4 + 9 + 21 + 4 + 6 + 2         # = 76
# Exponential time stepping adds per step: a quarter of a Philox block for
# the step lengths (15), one uniform (2), -log2 U with its clamp and the scale
# by ln 2 (3), the length into the noise scale (1) and into the drift (1).
OPS_EXPO_EXTRA = 15 + 2 + 3 + 1 + 1                           # = 22
# The Brownian-bridge test adds the distance test of a step pair's three
# points (9 per pair); with exponential steps also the pair's largest length
# into the cut distance sqrt(16.7 h) (3 per pair).
OPS_BRIDGE_EXTRA = 4.5
OPS_BRIDGE_EXPO_EXTRA = 1.5


# Drift evaluations other than the ring's 21: the tabulated density (cell
# coordinates, clamps and weights 10, the cell index 2, one 16-byte read, the
# two gradient components 2, the update 2) = 17.
DRIFT_OPS = {W.FAMILY_RING: 21, W.FAMILY_TABLE: 17}


def ops_per_step(stepper: int, exit_test: int, family: int = W.FAMILY_RING) -> float:
    ops = float(OPS_PER_STEP_RING_FP32) - DRIFT_OPS[W.FAMILY_RING] + DRIFT_OPS.get(family, 21)
    if stepper == W.STEP_EXPONENTIAL:
        ops += OPS_EXPO_EXTRA
    if exit_test == W.EXIT_BRIDGE:
        ops += OPS_BRIDGE_EXTRA + (OPS_BRIDGE_EXPO_EXTRA if stepper == W.STEP_EXPONENTIAL else 0)
    return ops
L2_BYTES = 129 * 1024 * 1024


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# DRAM bytes (read + write) of one launch of the path kernel at the 257 x 257
# ring workload with constant steps and the end-of-step test, from one ncu
# capture of the timed launch (dram__bytes_read.sum + dram__bytes_write.sum).
# Valid only for the kernel source it was taken on: the bench line reports
# null traffic once the source's SHA-256 differs.
PATH_KERNEL_TRAFFIC = {"bytes": 803840 + 512,
                       "source_sha256": "07474d4d0288ec637b6b0535bbccba9f6f5fc0cdf54897d7f3634b2386e0702a"}


# FP32 (FMA) pipe and issue-slot activity of the same kernel, from one ncu
# capture of the bench workload at N = 16384 (the same kernel, launch shape and
# chunking; sm__inst_executed_pipe_fma and smsp__issue_active, each as a share
# of its peak over the active cycles), keyed to the kernel source like the
# traffic: null once the source changes.
PATH_KERNEL_COUNTERS = {"fp32_fma_pipe": 0.3618, "issue_active": 0.7474,
                        "source_sha256": "07474d4d0288ec637b6b0535bbccba9f6f5fc0cdf54897d7f3634b2386e0702a"}


# The same counters for the kernel of the paper's stepper (exponential steps at
# lambda = 1e4 with the bridge test, the bench geometry), from one ncu capture
# at N = 16384 (same kernel and launch shape), with the share of lanes active
# per issued instruction (smsp__thread_inst_executed_per_inst_executed / 32).
PAPER_STEPPER_COUNTERS = {"fp32_fma_pipe": 0.3102, "issue_active": 0.7334,
                          "lanes_active": 21.86 / 32,
                          "source_sha256": "07474d4d0288ec637b6b0535bbccba9f6f5fc0cdf54897d7f3634b2386e0702a"}


def _mc_source_digest():
    import hashlib
    src = os.path.join(ROOT, "paper_1310_3435_gb300", "csrc", "mc.cu")
    try:
        with open(src, "rb") as fh:
            return hashlib.sha256(fh.read()).hexdigest()
    except OSError:
        return None


def _is_bench_workload(spec):
    return (spec.n, spec.sx, spec.family, spec.paths, spec.dt, spec.stepper,
            spec.exit_test) == (257, 4, W.FAMILY_RING, 100000, 1e-5, W.STEP_EULER,
                                W.EXIT_END_OF_STEP)


def path_kernel_traffic(spec):
    if _is_bench_workload(spec) and _mc_source_digest() == PATH_KERNEL_TRAFFIC["source_sha256"]:
        return PATH_KERNEL_TRAFFIC["bytes"]
    return None


def path_kernel_counters(spec):
    """(FP32 FMA-pipe fraction, issue-slot fraction) of the recorded capture,
    or (None, None) when it does not describe this workload and source."""
    c = PATH_KERNEL_COUNTERS
    if _is_bench_workload(spec) and _mc_source_digest() == c["source_sha256"]:
        return c["fp32_fma_pipe"], c["issue_active"]
    return None, None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled while the timed region
    runs (every 200 ms)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def make_spec(name: str):
    if name == "config1":
        return W.config1()
    if name == "config2":
        return W.config2()
    if name == "config4":
        return W.config4()
    raise ValueError(name)


def bench_spec(args, seed=None):
    """The workload of a single-mesh run with the command line's overrides
    (paths, mean step, stepper, exit test; `seed` for a replica's own seed)."""
    spec = make_spec(args.config)
    over = {}
    if seed is not None:
        over["seed"] = seed
    if args.paths:
        over["paths"] = args.paths
    if args.dt:
        over["dt"] = args.dt
    if args.stepper == "exponential":
        over["stepper"] = W.STEP_EXPONENTIAL
    if args.exit_test == "bridge":
        over["exit_test"] = W.EXIT_BRIDGE
    if args.table_tn:
        # a tabulated density in place of the analytic one: a seeded smooth
        # field of ln w on table_tn x table_tn nodes
        over["family"] = W.FAMILY_TABLE
        over["params"] = W.table_params(W.smooth_field(args.table_tn, seed=1, amplitude=2.0))
    spec = W.MeshSpec(**{**spec.__dict__, **over})
    if (spec.stepper != W.STEP_EULER or spec.exit_test != W.EXIT_END_OF_STEP or args.dt
            or args.table_tn):
        dens = "table %dx%d" % (args.table_tn, args.table_tn) if args.table_tn else ""
        spec = W.MeshSpec(**{**spec.__dict__, "label": "%s%s, %s steps, %s exit test, dt=%g" % (
            spec.label.split(" N=")[0].replace("ring", dens) if dens else spec.label.split(" N=")[0],
            "", args.stepper, args.exit_test, spec.dt)})
    return spec


# ------------------------------------------------------------ CPU oracle ----
def oracle_sample(spec, budget_s: float = 15.0, threads: int | None = None):
    """Times the FP64 oracle on a bounded sample of `spec`: evenly spaced
    interface nodes, the first paths of each node (the same Philox streams the
    GPU runs), sized to about `budget_s` seconds on the host cores."""
    import oracle
    threads = threads or oracle.default_threads()
    nodes = oracle.interface_nodes(spec.n, spec.sx, spec.sy)
    E = oracle.bmap_tables(spec.n, spec.bmap_mode, spec.family, spec.coef_mode, spec.params)
    k = max(threads, 1)
    idx = np.linspace(0, len(nodes) - 1, k).round().astype(int)
    # calibration: 32 paths per sampled node
    t0 = time.perf_counter()
    kw = dict(node_ids=idx, threads=threads, exit_test=spec.exit_test, stepper=spec.stepper)
    r = oracle.mc_nodes(spec.n, nodes[idx], E, spec.family, spec.coef_mode, spec.params,
                        spec.seed, 32, spec.dt, spec.cap(), spec.tie(), **kw)
    cal = time.perf_counter() - t0
    paths = int(max(32, min(spec.paths, 32 * budget_s / max(cal, 1e-3))))
    t0 = time.perf_counter()
    r = oracle.mc_nodes(spec.n, nodes[idx], E, spec.family, spec.coef_mode, spec.params,
                        spec.seed, paths, spec.dt, spec.cap(), spec.tie(), **kw)
    el = time.perf_counter() - t0
    steps = int(r["steps"].sum())
    return {"value": steps / el, "unit": "path-steps/s", "cores": threads, "kind": "oracle",
            "sample": "%d of %d interface nodes x %d paths (FP64, %d path-steps, %.1f s)"
                      % (len(idx), len(nodes), paths, steps, el),
            "seconds": el, "path_steps": steps,
            "_idx": idx, "_paths": paths, "_S": r["S_all"], "_Q": r["Q_all"],
            "_steps": r["steps"], "_ties": r["ties"]}


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    import oracle
    spec = bench_spec(args)
    threads = oracle.default_threads()
    for _ in range(args.warmup):
        oracle_sample(spec, budget_s=2.0, threads=threads)
    vals, secs, steps = [], 0.0, 0
    for _ in range(args.steps):
        s = oracle_sample(spec, budget_s=args.ref_budget, threads=threads)
        vals.append(s["value"])
        secs += s["seconds"]
        steps += s["path_steps"]
    value = steps / secs
    line = {"impl": "reference", "metric": "SDE path-steps/s", "value": value,
            "unit": "path-steps/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * secs / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": spec.label, "sample": s["sample"]},
            "cpu_baseline": {"value": value, "unit": "path-steps/s", "cores": threads,
                             "kind": "oracle", "sample": s["sample"]},
            "e2e": {"value": value, "unit": "path-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------ GPU arm ----
def run_native(args):
    import torch
    import torch.distributed as dist
    from paper_1310_3435_gb300 import native as N

    rank, world, local = env_rank()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # independent problem per rank: its own seed (weak scaling, no collective)
    from paper_1310_3435_gb300 import replicas
    spec = bench_spec(args, seed=replicas.rank_seed(make_spec(args.config).seed, rank))
    stream = torch.cuda.Stream(device=dev)
    plan = N.Plan(spec)
    mc = plan.mc_params(precision=spec.precision if args.precision is None else args.precision,
                        chunk=args.chunk)
    sp = plan.solve_params()
    n = spec.n
    mesh = torch.zeros((n, n, 2), dtype=torch.float64, device=dev)
    mean = torch.zeros((plan.n_nodes, 2), dtype=torch.float64, device=dev)
    se = torch.zeros((plan.n_nodes, 2), dtype=torch.float64, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def step(evs=None):
        if evs:
            evs[0].record(stream)
        N.sdd_interface_mc(plan.handle, mc, mean, se, want_stats=False, stream=stream)
        if evs:
            evs[1].record(stream)
        N.sdd_subdomain_solve(plan.handle, mean, sp, mesh, want_stats=False, stream=stream)
        if evs:
            evs[2].record(stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
            flush.zero_()
    torch.cuda.synchronize()
    mc_stats = N.sdd_plan_last_mc_stats(plan.handle)
    path_steps = int(mc_stats.path_steps)

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    sampler = ClockSampler(local)
    launches0 = N.sdd_kernel_launches()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    t_begin = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_begin.record(stream)
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            step(evs[k])
            flush.zero_()                      # L2 flush between timed steps
    t_end.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = N.sdd_kernel_launches() - launches0
    ms_mc = [e[0].elapsed_time(e[1]) for e in evs]
    ms_solve = [e[1].elapsed_time(e[2]) for e in evs]
    ms_step = [a + b for a, b in zip(ms_mc, ms_solve)]
    t_total = sum(ms_step) / 1000.0
    check = N.sdd_plan_last_mc_stats(plan.handle)
    assert int(check.path_steps) == path_steps
    t_total = replicas.max_over_ranks(t_total, device=dev)
    value = replicas.whole_job_rate(path_steps * args.steps, world, t_total)
    meshes_per_s = replicas.whole_job_rate(args.steps, world, t_total)

    # end to end through the public API with host buffers: plan (H2D of the
    # request's tables) + mesh generation + D2H of mesh and interface values
    e2e = None
    if not args.no_e2e:
        mesh_h = np.zeros((n, n, 2))
        mean_h = np.zeros((plan.n_nodes, 2))
        se_h = np.zeros((plan.n_nodes, 2))
        e2e_steps = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            with N.Plan(spec) as P2:
                N.sdd_mesh_generate(P2.handle, mc, sp, mesh_h, mean_h, se_h, want_stats=False,
                                    stream=stream)
        el = time.perf_counter() - t0
        h2d = plan.n_nodes * 2 * 4 + 8 * n * 8
        d2h = mesh_h.nbytes + mean_h.nbytes + se_h.nbytes
        e2e = {"value": world * path_steps * e2e_steps / el, "unit": "path-steps/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "meshes_per_s": world * e2e_steps / el}

    peaks, peak_kind = measured_peaks()
    sm_clock_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = sms * 128 * sm_clock_max * 1e6 / 1e9          # Gop/s
    t_mc = sum(ms_mc) / len(ms_mc) / 1000.0
    ops = ops_per_step(spec.stepper, spec.exit_test, spec.family)
    achieved = ops * path_steps / t_mc / 1e9
    line = {
        "mc_path_steps_per_s": achieved_steps_per_s(path_steps, t_mc),
        "metric": "SDE path-steps/s",
        "step": "one whole mesh generation: interface Monte Carlo + subdomain solves",
        "value": value, "unit": "path-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32-step/f64-acc" if mc.precision == N.SDD_FP32_STEP else "f64",
        "data": "synthetic",
        "config": {"workload": spec.label, "n": n, "split": [spec.sx, spec.sy],
                   "interface_nodes": plan.n_nodes, "paths_per_node": spec.paths,
                   "dt": spec.dt, "stepper": args.stepper, "exit_test": args.exit_test,
                   "path_steps_per_mesh": path_steps,
                   "l2": "flushed between timed steps (2x L2 write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "meshes_per_s": meshes_per_s,
        "ms_interface_mc": float(np.mean(ms_mc)), "ms_subdomain_solve": float(np.mean(ms_solve)),
        "max_stderr": float(mc_stats.max_stderr),
        "non_exits": int(mc_stats.non_exits),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Gop/s",
                     "frac": achieved / alu_peak, "traffic": path_kernel_traffic(spec),
                     "traffic_basis": "dram__bytes_read.sum + dram__bytes_write.sum of one "
                                      "launch (ncu), bytes; null if the kernel source changed",
                     "kernel": "k_paths<FP32, %s> (+k_reduce)" % (
                         "table" if spec.family == W.FAMILY_TABLE else "ring"),
                     "peak_basis": "%d SMs x 128 lanes x %.0f MHz (%s sm_max_mhz)"
                                   % (sms, sm_clock_max, peak_kind),
                     "ops_per_path_step": ops,
                     "fp32_fma_pipe_frac_ncu": path_kernel_counters(spec)[0],
                     "issue_frac_ncu": path_kernel_counters(spec)[1],
                     "pipe_basis": "ncu of the timed kernel source: FMA-pipe cycles and issue "
                                   "slots active over elapsed cycles; null if the source changed"},
        "clocks": clocks,
        "gpu_launches": int(launches),
    }
    if e2e:
        line["e2e"] = e2e
    line["mesh_quality"] = dict(mesh_quality_of(N, plan, mesh),
                                note="the timed mesh: at N = 1e5 the interface std-err exceeds the "
                                     "compressed spacing on the ring's flanks, so cells fold; the "
                                     "workload measures throughput, not a usable mesh")
    if not args.no_fp64:
        line["fp64_gpu"] = fp64_leg(N, spec, stream, dev, args.fp64_paths)
        line["fp32_over_fp64"] = line["fp64_gpu"]["comparable_value"] and (
            achieved_steps_per_s(path_steps, t_mc) / line["fp64_gpu"]["comparable_value"])
        line["fp64_gpu"]["equal_stderr"] = equal_stderr_leg(N, stream)
    if rank == 0 and not args.no_cpu:
        sample = oracle_sample(spec, budget_s=args.ref_budget)
        line["cpu_baseline"] = {k: v for k, v in sample.items()
                                if k in ("value", "unit", "cores", "kind", "sample")}
        line["precision_bias"] = precision_bias_leg(N, spec, sample, mc_stats.max_stderr, stream)
    plan.close()
    if rank == 0 and not args.no_paper_stepper:
        line["paper_stepper"] = paper_stepper_leg(N, spec, alu_peak, stream)
    if rank == 0 and not args.no_batched:
        line["batched"] = batched_leg(N, count=args.count)
        line["precision_stress"] = precision_stress_leg(N)
    if rank == 0 and not args.no_served:
        line["served"] = serve_leg(args.served_rates, args.served_count, args.served_stderr,
                                   1025, precision=W.FP32_STEP, ideal=True)
        # plain FP64 against mixed precision on one smaller stream (FP64 stepping
        # runs about 300x fewer path-steps/s): the same requests, both precisions
        small = dict(rates=[args.fp64_served_rate], count=args.fp64_served_count,
                     target_stderr=args.served_stderr, n_max=97)
        line["served_fp64"] = {"fp64": serve_leg(precision=W.FP64, **small),
                               "fp32_step_same_stream": serve_leg(precision=W.FP32_STEP, **small),
                               "note": "scaled down to n <= 97 so that FP64 stepping keeps up"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """Batched uneven meshes (256 meshes, n in {65..513}, splits 2..8, one
    bump each, 2e4 paths, dt = 5e-5): one C-ABI batch per step, replayed as a
    CUDA graph.  Prints one JSON line (path-steps/s and meshes/s)."""
    import torch
    from paper_1310_3435_gb300 import native as N
    torch.cuda.set_device(0)
    leg = batched_leg(N, count=args.count, paths=args.paths, autotune=not args.no_autotune,
                      steps=args.steps, warmup=args.warmup)
    line = {"metric": "SDE path-steps/s", "value": leg["path_steps_per_s"],
            "unit": "path-steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": leg["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32-step/f64-acc", "data": "synthetic",
            "config": {"workload": leg["workload"]}, "clocks": leg["clocks"],
            "gpu_launches": leg["gpu_launches"], "batched": leg}
    print(json.dumps(line))
    return 0


def run_serve(args):
    """Serving: Poisson stream of mesh requests (n log-uniform 65..n_max,
    splits 2..8, 1-3 bumps), paths per node chosen by a pilot for the std-err
    target, continuous batching; p50/p99 latency and meshes/s."""
    import torch
    torch.cuda.set_device(0)
    leg = serve_leg(args.rates, args.count, args.target_stderr, args.n_max,
                    precision=W.FP32_STEP if args.precision is None else args.precision,
                    max_batch=args.max_batch)
    print(json.dumps(dict({"metric": "served latency and meshes/s", "unit": "s"}, **leg)))
    return 0


def run_precision(args):
    """Precision report for a configuration (default config 4): FP32 stepping
    on the GPU against the FP64 oracle on an evenly spaced subsample of
    `sample_nodes` interface nodes, both replaying the same Philox streams of
    the first `sample_paths` paths (the paired difference is the
    precision-induced bias, separate from the Monte Carlo error), plus the
    GPU run at the configuration's full paths per node (std-err per node)."""
    import torch
    import oracle
    from paper_1310_3435_gb300 import native as N
    torch.cuda.set_device(0)
    spec = make_spec(args.config)
    nodes_all = oracle.interface_nodes(spec.n, spec.sx, spec.sy)
    m = len(nodes_all)
    idx = (np.arange(args.sample_nodes) * (m // args.sample_nodes)).astype(int)
    sub = W.MeshSpec(**{**spec.__dict__, "paths": args.sample_paths})
    out = {"metric": "precision report", "workload": spec.label, "interface_nodes": m,
           "sample": "%d nodes (every %d-th) x first %d paths" % (len(idx), m // len(idx),
                                                                  args.sample_paths)}
    with N.Plan(sub) as P:
        g32 = N.sdd_interface_mc_sums(P.handle, P.mc_params(precision=W.FP32_STEP))
    E = oracle.bmap_tables(spec.n, spec.bmap_mode, spec.family, spec.coef_mode, spec.params)
    t0 = time.perf_counter()
    o = oracle.mc_nodes(spec.n, nodes_all[idx], E, spec.family, spec.coef_mode, spec.params,
                        spec.seed, args.sample_paths, spec.dt, spec.cap(), 1e-11, node_ids=idx)
    t_or = time.perf_counter() - t0
    x0 = nodes_all[idx] / (spec.n - 1.0)
    Nn = float(args.sample_paths)
    m32 = x0 + g32["sum"][idx] / Nn
    mo = x0 + o["S_all"] / Nn
    se_o = np.sqrt(np.maximum(o["Q_all"] - o["S_all"] ** 2 / Nn, 0) / (Nn * (Nn - 1)))
    d = m32 - mo
    out["fp32_vs_fp64_oracle"] = {
        "max_abs": float(np.abs(d).max()), "mean_signed": float(d.mean()),
        "rms": float(np.sqrt((d ** 2).mean())),
        "max_abs_over_stderr": float((np.abs(d) / se_o).max()),
        "mc_stderr_median": float(np.median(se_o)), "mc_stderr_max": float(se_o.max()),
        "steps_rel_diff": float(abs(int(g32["steps"][idx].sum()) - int(o["steps"].sum()))
                                / o["steps"].sum()),
        "oracle_ties": int(o["ties"].sum()), "oracle_seconds": t_or}
    if not args.no_full:
        full = spec if not args.paths else W.MeshSpec(**{**spec.__dict__, "paths": args.paths})
        with N.Plan(full) as P:
            mean = torch.zeros((P.n_nodes, 2), dtype=torch.float64, device="cuda")
            se = torch.zeros((P.n_nodes, 2), dtype=torch.float64, device="cuda")
            stream = torch.cuda.Stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            N.sdd_interface_mc(P.handle, P.mc_params(), mean, se, want_stats=False, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            st = N.sdd_plan_last_mc_stats(P.handle)
            sec = e0.elapsed_time(e1) / 1000.0
            sec_np = se.cpu().numpy()
        out["full_run"] = {"paths_per_node": full.paths, "path_steps": int(st.path_steps),
                           "seconds": sec, "path_steps_per_s": st.path_steps / sec,
                           "stderr_max": float(sec_np.max()),
                           "stderr_median": float(np.median(sec_np)),
                           "non_exits": int(st.non_exits)}
    print(json.dumps(out))
    return 0


def five_ring_ln_rho(tn: int, alpha: float = 0.2, R: float = 30.0) -> np.ndarray:
    """ln of the paper's five-ring arc-length monitor (eq. FiveRingMonitorFunction,
    rho = sqrt(1 + alpha |grad u|^2), u a sum of five tanh rings on [-1,1]^2) at
    the tn x tn nodes of the unit square, through x = 2s - 1, y = 2t - 1."""
    g = np.arange(tn) / (tn - 1.0)
    S, T = np.meshgrid(g, g, indexing="xy")
    x, y = 2.0 * S - 1.0, 2.0 * T - 1.0
    ux = np.zeros_like(x)
    uy = np.zeros_like(x)
    for cx, cy in ((0.0, 0.0), (0.5, 0.5), (0.5, -0.5), (-0.5, 0.5), (-0.5, -0.5)):
        q = (x - cx) ** 2 + (y - cy) ** 2 - 0.125
        sech2 = 1.0 / np.cosh(R * q) ** 2
        ux += R * sech2 * 2.0 * (x - cx)
        uy += R * sech2 * 2.0 * (y - cy)
    return 0.5 * np.log1p(alpha * (ux * ux + uy * uy))


def huang_sloan_ln_rho(tn: int, alpha: float = 0.7, R: float = 15.0) -> np.ndarray:
    """ln of the Huang-Sloan monitor of §4 (eq. HuangSloanMonitorFunction): the
    arc-length monitor rho = sqrt(1 + alpha |grad u|^2) of the boundary layer
    u = (1 - exp(R (x - 1))) sin(pi y) on the unit square, at its tn x tn nodes
    (row b = y = b / (tn - 1))."""
    g = np.arange(tn) / (tn - 1.0)
    x, y = np.meshgrid(g, g, indexing="xy")
    e = np.exp(R * (x - 1.0))
    ux = -R * e * np.sin(np.pi * y)
    uy = np.pi * (1.0 - e) * np.cos(np.pi * y)
    return 0.5 * np.log1p(alpha * (ux * ux + uy * uy))


# The Mackenzie front of §4 (eq. MackenzieMonitorFunction, alpha = 10, R = 50):
# rho = 1 / (1 + alpha exp(-R (y - 1/2 - sin(2 pi x) / 4)^2)), so the
# generator's coefficient 1/rho is the RIDGE family with these parameters.
MACKENZIE_RIDGE = (10.0, 50.0, 0.5, 0.25, 1.0)


def run_paper_performance(args):
    """The paper's performance study (§5) in its workload shape on one GB300:
    the five-ring arc-length monitor (tabulated on 1025 x 1025 nodes, w =
    1/rho), exponential steps with the boundary test at the paper's lambda =
    1000 on [-1,1]^2 (mean step 1/(4 lambda) on the unit square), FP32
    stepping, CG + FP64 refinement.  T_stoc and T_sub per mesh are CUDA-event
    medians after a warm-up, beside the paper's 16-core times:
      * Table 5: 4 x 4 subdomains, n = 37 ... 197, N = 5000, Monte Carlo at
        every interface node and at the extrema placement;
      * Tables 6 and 7: 157^2, 4 x 4, extrema placement, N = 500 ... 5000,
        R against the single-domain mesh without and with smoothing on the
        subdomains (5 steps, k = 1000, the largest stable FTCS step dt =
        h^2 / 4: the paper's dt = 1e-4 is unstable on this grid; the paper
        also smoothed the interface values with a third-party routine, which
        is not reproduced);
      * Table 8: 197^2, S = 2 x 2, 3 x 3, 4 x 4, extrema placement, N = 5000,
        with T_1, the single-domain solve."""
    import torch
    from paper_1310_3435_gb300 import native as N
    torch.cuda.set_device(0)
    params = W.table_params(five_ring_ln_rho(1025))
    stream = torch.cuda.Stream()

    def spec_of(n, s, paths):
        return W.MeshSpec(n=n, sx=s, sy=s, family=W.FAMILY_TABLE, params=params,
                          coef_mode=W.COEF_INV_W, bmap_mode=W.BMAP_PAPER_1D, paths=paths,
                          dt=1.0 / 4000.0, precision=W.FP32_STEP, stepper=W.STEP_EXPONENTIAL,
                          exit_test=W.EXIT_BRIDGE, solver=W.SOLVER_CG_FP32_REFINE, tol=1e-10)

    def timed(P, place, reps=4, smooth_steps=0):
        """Median T_stoc, T_sub (and T_smooth) over reps - 1 runs after a
        warm-up; returns the times, the last mesh (host) and the MC stats."""
        N.sdd_plan_set_placement(P.handle, place, 0)
        mean = torch.zeros((P.n_nodes, 2), dtype=torch.float64, device="cuda")
        mesh = torch.zeros((P.n, P.n, 2), dtype=torch.float64, device="cuda")
        mc, sp = P.mc_params(), P.solve_params()
        h = 1.0 / (P.n - 1)
        t = {"mc": [], "sub": [], "smooth": []}
        for rep in range(reps):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            e[0].record(stream)
            N.sdd_interface_mc(P.handle, mc, mean, None, want_stats=False, stream=stream)
            e[1].record(stream)
            N.sdd_subdomain_solve(P.handle, mean, sp, mesh, want_stats=False, stream=stream)
            e[2].record(stream)
            if smooth_steps:
                N.sdd_mesh_smooth_subdomains(P.handle, mesh, smooth_steps, 0.25 * h * h, 1000.0,
                                             False, stream=stream)
            e[3].record(stream)
            stream.synchronize()
            if rep:                                   # the first run warms up
                t["mc"].append(e[0].elapsed_time(e[1]) / 1000.0)
                t["sub"].append(e[1].elapsed_time(e[2]) / 1000.0)
                t["smooth"].append(e[2].elapsed_time(e[3]) / 1000.0)
        st = N.sdd_plan_last_mc_stats(P.handle)
        return ({k: float(np.median(v)) for k, v in t.items()}, mesh.cpu().numpy(), st)

    def single_domain(n, reps=4):
        """The single-domain mesh and its solve time T_1 (median after a warm-up)."""
        with N.Plan(spec_of(n, 1, 2)) as P:
            ref = torch.zeros((n, n, 2), dtype=torch.float64, device="cuda")
            sp = P.solve_params()
            ts = []
            for rep in range(reps):
                e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                e[0].record(stream)
                N.sdd_subdomain_solve(P.handle, None, sp, ref, want_stats=False, stream=stream)
                e[1].record(stream)
                stream.synchronize()
                if rep:
                    ts.append(e[0].elapsed_time(e[1]) / 1000.0)
            return ref.cpu().numpy(), float(np.median(ts))

    def r_of(P, mesh, ref):
        q = N.sdd_mesh_quality(P.handle, mesh, ref)
        return {"R_max": q["r_max"], "R_mean": q["r_mean"], "folds": q["folds"]}

    # Table 5
    paper5 = {37: (5.47, 0.00), 77: (7.56, 0.02), 117: (8.81, 0.08), 157: (8.88, 0.21),
              197: (9.06, 0.47)}
    rows = []
    for n in (37, 77, 117, 157, 197):
        for place in (N.SDD_PLACE_ALL, N.SDD_PLACE_EXTREMA):
            with N.Plan(spec_of(n, 4, 5000)) as P:
                t, _, st = timed(P, place)
                _, n_mc = N.sdd_plan_placement(P.handle)
            rows.append({"n": n, "placement": "all" if place == N.SDD_PLACE_ALL else "extrema",
                         "mc_nodes": n_mc, "path_steps": int(st.path_steps),
                         "T_stoc_s": t["mc"], "T_sub_s": t["sub"],
                         "paper_T_stoc_s": paper5[n][0], "paper_T_sub_s": paper5[n][1],
                         "non_exits": int(st.non_exits)})
    # Tables 6 and 7
    paper67 = {500: (0.04, 0.96, 0.46, 0.98, 0.91), 1000: (0.24, 0.98, 0.82, 0.99, 1.88),
               2000: (0.71, 1.0, 0.96, 1.0, 3.68), 5000: (0.93, 1.0, 0.98, 1.0, 9.07)}
    ref157, _ = single_domain(157)
    rows67 = []
    for paths in (500, 1000, 2000, 5000):
        with N.Plan(spec_of(157, 4, paths)) as P:
            t, mesh, st = timed(P, N.SDD_PLACE_EXTREMA, smooth_steps=5)
            # the timed runs end smoothed: the same mesh once more without smoothing
            plain = np.zeros_like(mesh)
            N.sdd_mesh_generate(P.handle, P.mc_params(), P.solve_params(), plain)
            r0 = r_of(P, plain, ref157)
            r1 = r_of(P, mesh, ref157)
        pr = paper67[paths]
        rows67.append({"N": paths, "no_smoothing": r0, "subdomain_smoothing": r1,
                       "T_stoc_s": t["mc"], "T_sub_s": t["sub"], "T_smooth_s": t["smooth"],
                       "path_steps": int(st.path_steps),
                       "paper": {"R_max": pr[0], "R_mean": pr[1], "R_max_smoothed": pr[2],
                                 "R_mean_smoothed": pr[3], "T_stoc_s": pr[4], "T_sub_s": 0.21,
                                 "T_smooth_s": 0.01}})
    # Table 8
    paper8 = {2: (0.96, 12.54, 14.89), 3: (0.89, 10.81, 2.95), 4: (0.96, 10.59, 0.46)}
    ref197, t1 = single_domain(197)
    rows8 = []
    for s in (2, 3, 4):
        with N.Plan(spec_of(197, s, 5000)) as P:
            t, mesh, st = timed(P, N.SDD_PLACE_EXTREMA)
            _, n_mc = N.sdd_plan_placement(P.handle)
            r = r_of(P, mesh, ref197)
        rows8.append({"S": s * s, "mc_nodes": n_mc, **r, "T_stoc_s": t["mc"], "T_sub_s": t["sub"],
                      "T_total_s": t["mc"] + t["sub"], "T_1_s": t1,
                      "paper": {"R_max": paper8[s][0], "T_stoc_s": paper8[s][1],
                                "T_sub_s": paper8[s][2], "T_1_s": 64.0}})
    print(json.dumps({"metric": "T_stoc, T_sub of the paper's performance study (Tables 5-8 shape)",
                      "workload": "five-ring arc-length monitor (table 1025^2), N=5000 unless "
                                  "stated, exponential steps lambda=1000 on [-1,1]^2, boundary "
                                  "test, FP32",
                      "paper_hardware": "16-core CPU machine (the paper's §5)",
                      "rows": rows, "table6_7_157": rows67, "table8_197": rows8}))
    return 0


def run_quality(args):
    """Mesh-quality report on the paper's running example (eq.
    MonitorFunctionRunningExample: rho = 1 + 15 exp(-50 (x - 3/4)^2 - 50 (y -
    1/2)^2 - 1/2), generator coefficient 1/rho, 29 x 29 grid, the 1D generator
    on the sides as boundary map, §3.2), with exponential time stepping and
    the boundary test as in the paper's experiments.  Against the
    single-domain mesh (Q_max, Q_mean, R_max, R_mean, l_inf; §3.1, §3.3):
      * the fully probabilistic mesh (§3.3) at lambda = 1000, N = 1000 and
        10000, and the N = 1000 mesh after m = 1, 2, 5, 10 Perona-Malik steps
        (dt = 1e-4, k = 1000, §3.4; the reference smoothed alike);
      * the 2 x 2 stochastic-deterministic mesh at lambda = 1 / quality-dt,
        N = 1e3, 1e4, 1e5, with every interface node, 7 equispaced points per
        line, or the extrema placement (§3.5, §3.6);
      * §4's further examples on the same grid, 2 x 2 with every interface
        node: the Huang-Sloan monitor, and the Mackenzie front in the shape of
        Tables 3 and 4 with global, per-subdomain and shifted-subdomain
        smoothing, each against its own single-domain mesh."""
    import torch
    from paper_1310_3435_gb300 import native as N
    torch.cuda.set_device(0)
    n = 29
    rho = W.bumps((15.0 * math.exp(-0.5), 0.75, 0.5, 50.0, 50.0))
    base = dict(n=n, family=W.FAMILY_BUMPS, params=rho, coef_mode=W.COEF_INV_W,
                bmap_mode=W.BMAP_PAPER_1D, seed=0, precision=W.FP32_STEP,
                exit_test=W.EXIT_BRIDGE, stepper=W.STEP_EXPONENTIAL, solver=W.SOLVER_SOR,
                tol=1e-12)
    single = W.MeshSpec(sx=1, sy=1, paths=2, dt=1e-3, **base)
    with N.Plan(single) as P:
        ref = np.zeros((n, n, 2))
        N.sdd_subdomain_solve(P.handle, np.zeros((0, 2)), P.solve_params(), ref)
        q_ref = N.sdd_mesh_quality(P.handle, ref)

    def row(P, mesh, against, **extra):
        q = N.sdd_mesh_quality(P.handle, mesh, against)
        out = dict(extra)
        out.update({k: q[k] for k in ("q_max", "q_mean", "ref_q_max", "ref_q_mean", "r_max",
                                      "r_mean", "l_inf", "folds")})
        return out

    full = []
    for paths in (1000, 10000):
        spec = W.MeshSpec(sx=n - 1, sy=n - 1, paths=paths, dt=1e-3, **base)
        with N.Plan(spec) as P:
            mesh = np.zeros((n, n, 2))
            ms, _ = N.sdd_mesh_generate(P.handle, P.mc_params(), P.solve_params(), mesh)
            full.append(row(P, mesh, ref, N=paths, m=0, path_steps=int(ms.path_steps)))
            if paths == 1000:
                for m in (1, 2, 5, 10):
                    sm, rs = mesh.copy(), ref.copy()
                    N.sdd_mesh_smooth(P.handle, sm, m, 1e-4, 1000.0)
                    N.sdd_mesh_smooth(P.handle, rs, m, 1e-4, 1000.0)
                    full.append(row(P, sm, rs, N=paths, m=m))
    dd = []
    for paths in (1000, 10000, 100000):
        for place, k in ((N.SDD_PLACE_ALL, 0), (N.SDD_PLACE_EQUISPACED, 7),
                         (N.SDD_PLACE_EXTREMA, 0)):
            spec = W.MeshSpec(sx=2, sy=2, paths=paths, dt=args.quality_dt, **base)
            with N.Plan(spec) as P:
                N.sdd_plan_set_placement(P.handle, place, k)
                mesh = np.zeros((n, n, 2))
                ms, _ = N.sdd_mesh_generate(P.handle, P.mc_params(), P.solve_params(), mesh)
                _, n_mc = N.sdd_plan_placement(P.handle)
                dd.append(row(P, mesh, ref, N=paths,
                              placement=["all", "7 equispaced", "extrema"][place],
                              mc_nodes=n_mc, path_steps=int(ms.path_steps)))
    # §4's further examples, 2 x 2 with every interface node, each against its
    # own single-domain mesh: the Huang-Sloan monitor (tabulated ln rho on
    # 257^2 nodes, coefficient 1/rho) at N = 1e4, lambda = 1e3 and 1e4; the
    # Mackenzie front (coefficient 1/rho = the ridge) in the shape of the
    # paper's Tables 3 (N = 1e4, lambda = 1e3 .. 1e4) and 4 (lambda = 5e3, N =
    # 1e3 .. 1e4), without smoothing, with 5 Perona-Malik steps (dt = 1e-4,
    # k = 1000) on the whole mesh, on each subdomain, and on each subdomain and
    # then on the shifted subdomains; the reference of the smoothed rows is the
    # single-domain mesh smoothed on the whole square, as in the paper's tables
    further = []
    m, sdt, sk = 5, 1e-4, 1000.0
    for name, fam, params, mode, runs in (
            ("Huang-Sloan", W.FAMILY_TABLE, W.table_params(huang_sloan_ln_rho(257)), W.COEF_INV_W,
             ((1e3, 10000), (1e4, 10000))),
            ("Mackenzie", W.FAMILY_RIDGE, MACKENZIE_RIDGE, W.COEF_W,
             tuple((lam, 10000) for lam in (1e3, 2e3, 5e3, 1e4)) +
             tuple((5e3, paths) for paths in (1000, 2000, 5000)))):
        ex = dict(base, family=fam, params=params, coef_mode=mode)
        with N.Plan(W.MeshSpec(sx=1, sy=1, paths=2, dt=1e-3, **ex)) as P:
            ref_ex = np.zeros((n, n, 2))
            N.sdd_subdomain_solve(P.handle, np.zeros((0, 2)), P.solve_params(), ref_ex)
            ref_sm = ref_ex.copy()
            N.sdd_mesh_smooth(P.handle, ref_sm, m, sdt, sk)
        for lam, paths in runs:
            spec = W.MeshSpec(sx=2, sy=2, paths=paths, dt=1.0 / lam, **ex)
            with N.Plan(spec) as P:
                mesh = np.zeros((n, n, 2))
                ms, _ = N.sdd_mesh_generate(P.handle, P.mc_params(), P.solve_params(), mesh)
                info = dict(monitor=name, N=paths, lam=lam, path_steps=int(ms.path_steps))
                further.append(row(P, mesh, ref_ex, smoothing="none", **info))
                if name != "Mackenzie":
                    continue
                g = mesh.copy()
                N.sdd_mesh_smooth(P.handle, g, m, sdt, sk)
                further.append(row(P, g, ref_sm, smoothing="global", **info))
                sub = mesh.copy()
                N.sdd_mesh_smooth_subdomains(P.handle, sub, m, sdt, sk, False)
                further.append(row(P, sub, ref_sm, smoothing="subdomains", **info))
                N.sdd_mesh_smooth_subdomains(P.handle, sub, m, sdt, sk, True)
                further.append(row(P, sub, ref_sm, smoothing="subdomains, then shifted", **info))
    print(json.dumps({"metric": "mesh quality vs single-domain mesh",
                      "workload": "running example, 29x29, 1D boundary map, exponential steps "
                                  "with the boundary test",
                      "single_domain": {"q_max": q_ref["q_max"], "q_mean": q_ref["q_mean"]},
                      "fully_probabilistic": {"lambda": 1000, "smoothing": "dt=1e-4, k=1000",
                                              "rows": full},
                      "dd_2x2": {"lambda": 1.0 / args.quality_dt, "rows": dd},
                      "further_examples_2x2": {"grid": "29x29, every interface node",
                                               "smoothing": "%d steps, dt=%g, k=%g" % (m, sdt, sk),
                                               "rows": further}}))
    return 0


def achieved_steps_per_s(path_steps, seconds):
    return path_steps / seconds


def fp64_leg(N, spec, stream, dev, paths):
    """Plain FP64 stepping on the GPU, same workload geometry and streams, on
    the first `paths` paths of every node (FP64 is far slower on this part):
    the interface Monte Carlo's path-steps/s, comparable with the FP32 path
    kernel's rate (path-steps/s is per unit of work)."""
    import torch
    sub = W.MeshSpec(**{**spec.__dict__, "paths": paths, "precision": W.FP64})
    with N.Plan(sub) as P:
        mc = P.mc_params()
        N.sdd_interface_mc(P.handle, mc, want_stats=False, stream=stream)      # warm-up
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        N.sdd_interface_mc(P.handle, mc, want_stats=False, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        st = N.sdd_plan_last_mc_stats(P.handle)
        sec = e0.elapsed_time(e1) / 1000.0
    return {"paths_per_node": paths, "path_steps": int(st.path_steps), "seconds": sec,
            "comparable_value": st.path_steps / sec, "unit": "path-steps/s",
            "note": "interface Monte Carlo only, FP64 stepping"}


# Algorithmic bytes of one multigrid-preconditioned FP32 CG iteration per
# interior node of level 0 (float2 values of both components, FP32
# coefficients): the operator product (read p and two edge coefficients per
# node, write q: 8 + 8 + 8), the x and r updates (read p q x r, write x r:
# 48), the red-black sweeps before and after the coarse correction (read r,
# z, two coefficients, 1/diag, write z: 36 each, 72), the residual (read r z
# and the coefficients, write t: 32), the restriction (read t: 8), the
# prolongation (read and write z: 16), r.z (16) and the p update (read z p,
# write p: 24).  The coarse levels add under a third of the V-cycle's bytes
# and are not counted.
SOLVE_BYTES_PER_NODE_ITERATION = 24 + 48 + 72 + 32 + 8 + 16 + 16 + 24     # = 240


def precision_bias_leg(N, spec, sample, timed_max_stderr, stream):
    """The precision-induced bias of the timed result, apart from its Monte
    Carlo error: the GPU path in the timed precision on the cpu_baseline's
    oracle sample (the same nodes and the same first paths, i.e. the same
    Philox streams), paired with the FP64 oracle node by node."""
    idx, paths = sample["_idx"], int(sample["_paths"])
    sub = W.MeshSpec(**{**spec.__dict__, "paths": paths})
    with N.Plan(sub) as P:
        g = N.sdd_interface_mc_sums(P.handle, P.mc_params(precision=spec.precision), stream=stream)
    S_o, Q_o = sample["_S"], sample["_Q"]
    Nn = float(paths)
    d = (g["sum"][idx] - S_o) / Nn                     # paired difference of the means
    se_o = np.sqrt(np.maximum(Q_o - S_o ** 2 / Nn, 0.0) / (Nn * (Nn - 1.0)))
    steps_o = int(np.asarray(sample["_steps"]).sum())
    return {"sample": "%d nodes x first %d paths, the cpu_baseline's sample" % (len(idx), paths),
            "max_abs": float(np.abs(d).max()), "mean_signed": float(d.mean()),
            "max_abs_over_stderr": float((np.abs(d) / np.maximum(se_o, 1e-300)).max()),
            "sample_stderr_max": float(se_o.max()),
            "steps_rel_diff": abs(int(g["steps"][idx].sum()) - steps_o) / max(steps_o, 1),
            "oracle_ties": int(np.asarray(sample["_ties"]).sum()),
            "timed_result_max_stderr": float(timed_max_stderr),
            "note": "GPU (timed precision) minus the FP64 oracle on identical streams: "
                    "precision-induced bias; the timed result's Monte Carlo std-err beside it"}


def bias_on_sample(N, specs, nodes_per_mesh=8, paths=2048):
    """Precision-induced bias of FP32 stepping on a sample: for each mesh, evenly
    spaced interface nodes, the first `paths` paths of each on the GPU (the
    timed precision) and in the FP64 oracle, the same Philox streams."""
    import oracle
    worst, worst_sigma, signed, count = 0.0, 0.0, 0.0, 0
    for spec in specs:
        sub = W.MeshSpec(**{**spec.__dict__, "paths": paths})
        nodes = oracle.interface_nodes(sub.n, sub.sx, sub.sy)
        idx = np.linspace(0, len(nodes) - 1, min(nodes_per_mesh, len(nodes))).round().astype(int)
        with N.Plan(sub) as P:
            g = N.sdd_interface_mc_sums(P.handle, P.mc_params())
        E = oracle.bmap_tables(sub.n, sub.bmap_mode, sub.family, sub.coef_mode, sub.params)
        o = oracle.mc_nodes(sub.n, nodes[idx], E, sub.family, sub.coef_mode, sub.params, sub.seed,
                            paths, sub.dt, sub.cap(), 1e-11, node_ids=idx,
                            exit_test=sub.exit_test, stepper=sub.stepper)
        d = (g["sum"][idx] - o["S_all"]) / float(paths)
        se = np.sqrt(np.maximum(o["Q_all"] - o["S_all"] ** 2 / paths, 0) / (paths * (paths - 1.0)))
        worst = max(worst, float(np.abs(d).max()))
        worst_sigma = max(worst_sigma, float((np.abs(d) / np.maximum(se, 1e-300)).max()))
        signed += float(d.sum())
        count += d.size
    return {"sample": "%d meshes x %d nodes x first %d paths" % (len(specs), nodes_per_mesh, paths),
            "max_abs": worst, "max_abs_over_stderr": worst_sigma, "mean_signed": signed / count}


def precision_stress_leg(N, paths=20000, stream=None):
    """The precision-stress workload (1025 x 1025, 8 x 8, the anisotropic
    ridge, dt = 1e-5, FP32 stepping with FP64 sums) at a reduced N, one
    single-mesh launch timed with CUDA events after a warm-up, with the
    precision-induced bias on a 64-node oracle sample beside its Monte Carlo
    error."""
    import torch
    spec = W.config4(paths=paths)
    stream = stream or torch.cuda.Stream()
    with N.Plan(spec) as P:
        mc = P.mc_params()
        mean = torch.zeros((P.n_nodes, 2), dtype=torch.float64, device="cuda")
        se = torch.zeros_like(mean)
        N.sdd_interface_mc(P.handle, P.mc_params(paths=1024), mean, se, want_stats=False,
                           stream=stream)                                  # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        N.sdd_interface_mc(P.handle, mc, mean, se, want_stats=False, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        st = N.sdd_plan_last_mc_stats(P.handle)
        sec = e0.elapsed_time(e1) / 1000.0
    return {"workload": "1025x1025 8x8 ridge w = 1 + 20 exp(-200 (t - 0.3 - 0.2 sin 2 pi s)^2), "
                        "dt=1e-5, FP32 stepping, N=%d (the configuration's 1e6 scaled down)" % paths,
            "interface_nodes": int(P.n_nodes), "path_steps": int(st.path_steps), "seconds": sec,
            "path_steps_per_s": st.path_steps / sec, "max_stderr": float(st.max_stderr),
            "non_exits": int(st.non_exits),
            "precision_bias": bias_on_sample(N, [spec], nodes_per_mesh=64, paths=2048)}


def paper_stepper_leg(N, spec, alu_peak, stream, lam=1e4, reps=3):
    """The paper's own stepper on the timed geometry: exponential time
    stepping at lambda = 1e4 (mean step 1e-4) with the Brownian-bridge
    boundary test, FP32 stepping with FP64 sums, the same N.  One warm-up
    launch, then the median of `reps` CUDA-event timed launches of the
    interface Monte Carlo; its ALU roofline at the stepper's operation count."""
    import torch
    ps = W.MeshSpec(**{**spec.__dict__, "stepper": W.STEP_EXPONENTIAL,
                       "exit_test": W.EXIT_BRIDGE, "dt": 1.0 / lam})
    with N.Plan(ps) as P:
        mc = P.mc_params()
        N.sdd_interface_mc(P.handle, mc, want_stats=False, stream=stream)
        ms = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            N.sdd_interface_mc(P.handle, mc, want_stats=False, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        st = N.sdd_plan_last_mc_stats(P.handle)
    t = sorted(ms)[len(ms) // 2] / 1000.0
    ops = ops_per_step(ps.stepper, ps.exit_test, ps.family)
    achieved = ops * st.path_steps / t / 1e9
    c = PAPER_STEPPER_COUNTERS
    known = (ps.n, ps.sx, ps.family, ps.paths) == (257, 4, W.FAMILY_RING, 100000) and \
        _mc_source_digest() == c["source_sha256"]
    return {"workload": "%dx%d %dx%d ring N=%d, exponential steps lambda=%g (mean step %g), "
                        "Brownian-bridge test" % (ps.n, ps.n, ps.sx, ps.sy, ps.paths, lam, ps.dt),
            "path_steps_per_s": st.path_steps / t, "ms_interface_mc": 1000.0 * t,
            "steps_per_path": st.path_steps / max(st.paths, 1),
            "max_stderr": float(st.max_stderr), "non_exits": int(st.non_exits),
            "l2": "not flushed (a launch reads under 1 MB of tables and node lists)",
            "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak,
                         "unit": "Gop/s", "frac": achieved / alu_peak,
                         "ops_per_path_step": ops,
                         "fp32_fma_pipe_frac_ncu": c["fp32_fma_pipe"] if known else None,
                         "issue_frac_ncu": c["issue_active"] if known else None,
                         "lanes_active_frac_ncu": c["lanes_active"] if known else None,
                         "pipe_basis": "ncu of the kernel source at N = 16384; null if the "
                                       "source or the geometry changed"}}


def mesh_quality_of(N, plan, mesh):
    """Q_max, Q_mean and folded cells of a generated mesh (k_quality)."""
    q = N.sdd_mesh_quality(plan.handle, mesh)
    return {"q_max": q["q_max"], "q_mean": q["q_mean"], "folds": int(q["folds"])}


def equal_stderr_leg(N, stream, reps=3):
    """Plain FP64 against mixed precision at equal statistical accuracy: the
    33 x 33, 2 x 2 bump workload at N = 4000, dt = 1e-4 (the same Philox
    streams, so the same Monte Carlo error), one whole mesh generation each:
    FP64 stepping + FP64 SOR, and FP32 stepping (FP64 sums) + FP32 CG with
    FP64 refinement, both to 1e-10.  CUDA-event timed, median of `reps`
    after a warm-up."""
    import torch
    spec = W.config1()
    out = {"workload": spec.label + ", whole mesh generation", "reps": reps}
    for name, prec, solver in (("fp64", W.FP64, W.SOLVER_SOR),
                               ("fp32_step", W.FP32_STEP, W.SOLVER_CG_FP32_REFINE)):
        with N.Plan(spec) as P:
            mesh = torch.zeros((spec.n, spec.n, 2), dtype=torch.float64, device="cuda")
            mc = P.mc_params(precision=prec)
            sp = P.solve_params(solver=solver)
            N.sdd_mesh_generate(P.handle, mc, sp, mesh, want_stats=False, stream=stream)
            ms = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                N.sdd_mesh_generate(P.handle, mc, sp, mesh, want_stats=False, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            st = N.sdd_plan_last_mc_stats(P.handle)
            t = float(np.median(ms)) / 1000.0
            out[name] = {"meshes_per_s": 1.0 / t, "ms_per_mesh": 1000.0 * t,
                         "path_steps_per_s": st.path_steps / t, "max_stderr": st.max_stderr,
                         "solver": "SOR FP64" if solver == W.SOLVER_SOR else "CG FP32 + FP64 refinement"}
    out["fp32_over_fp64_meshes_per_s"] = out["fp32_step"]["meshes_per_s"] / out["fp64"]["meshes_per_s"]
    return out


def batched_leg(N, count=256, paths=0, autotune=True, steps=1, warmup=1, stream=None):
    """Batched uneven meshes (n in {65..513}, splits 2..8, one bump each,
    N = 2e4, dt = 5e-5): one C-ABI batch, replayed as a CUDA graph, timed
    with CUDA events (L2 flushed between timed runs); then the fill + solve
    phase alone (from the interface values in place)."""
    import torch
    specs = W.config3(count=count)
    if paths:
        specs = [W.MeshSpec(**{**sp.__dict__, "paths": paths}) for sp in specs]
    plans = [N.Plan(sp) for sp in specs]
    stream = stream or torch.cuda.Stream()
    tuned = None
    mcs = [p.mc_params() for p in plans]
    sps = [p.solve_params() for p in plans]
    if autotune:
        from paper_1310_3435_gb300 import autotune as AT
        t0 = time.perf_counter()
        tuner = AT.Autotuner()
        picks = [tuner.tune(sp, p.n_nodes) for sp, p in zip(specs, plans)]
        tuner.save()
        mcs = [p.mc_params(chunk=k["chunk"]) for p, k in zip(plans, picks)]
        sps = [p.solve_params(block_threads=k["block_threads"]) for p, k in zip(plans, picks)]
        # the batch's one solve launch: its own CTA size, timed on the whole batch
        # (the interface values: a first Monte Carlo-free solve from the boundary
        # map is enough, the solve's cost does not depend on them)
        bt = tuner.tune_batch_solve(plans, mcs, sps)
        sps = [p.solve_params(block_threads=bt) for p in plans]
        tuned = {"buckets_timed": tuner.timed, "seconds": time.perf_counter() - t0,
                 "block_threads_per_bucket": sorted({k["block_threads"] for k in picks}),
                 "batch_solve_block_threads": bt,
                 "chunks": sorted({k["chunk"] for k in picks})}
    t0 = time.perf_counter()
    batch = N.Batch(plans, mcs, sps)
    t_create = time.perf_counter() - t0
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        batch.run(use_graph=True, stream=stream)
    stream.synchronize()
    launches0 = N.sdd_kernel_launches()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.zero_()
            evs[k][0].record(stream)
            batch.run(use_graph=True, stream=stream)
            evs[k][1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = N.sdd_kernel_launches() - launches0
    t = sum(a.elapsed_time(b) for a, b in evs) / 1000.0
    path_steps, solve_ok, max_se, max_iter = 0, 0, 0.0, 0
    for i in range(len(plans)):
        ms, ss = batch.stats(i, allow_not_converged=True)
        path_steps += int(ms.path_steps)
        solve_ok += int(ss.converged == ss.subdomains)
        max_se = max(max_se, float(ms.max_stderr))
        max_iter = max(max_iter, int(ss.max_iterations))

    def solve_phase(b):
        """The fill + solve phase alone, from the interface values in place."""
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush.zero_()
            e0.record(stream)
            b.run_phases(2, stream=stream)
            e1.record(stream)
        torch.cuda.synchronize()
        work, its, ok = 0.0, 0, 0
        for i in range(len(plans)):
            _, ss = b.stats(i, allow_not_converged=True)
            work += ss.node_iterations
            its = max(its, int(ss.max_iterations))
            ok += int(ss.converged == ss.subdomains)
        return e0.elapsed_time(e1), work, its, ok

    ms_solve, node_its, _, _ = solve_phase(batch)
    # the same solves with the diagonal (Jacobi) preconditioner, for comparison
    # (CTAs of 1024 threads, its fastest size on this batch)
    jac = N.Batch(plans, mcs, [p.solve_params(solver=W.SOLVER_CG_JACOBI_FP32_REFINE,
                                              block_threads=1024) for p in plans])
    solve_phase(jac)                                  # warm-up
    ms_jac, node_its_jac, its_jac, ok_jac = solve_phase(jac)
    jac.close()
    grid_nodes = sum(p.n * p.n for p in plans)
    nodes = sum(p.n_nodes for p in plans)
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    solve_bytes = SOLVE_BYTES_PER_NODE_ITERATION * node_its
    solve_gbs = solve_bytes / (ms_solve / 1000.0) / 1e9
    out = {"workload": "batched uneven: %d meshes, n in {65,129,257,513}, splits 2..8, 1 bump, "
                       "N=%d, dt=5e-5, one CUDA-graph replay per step" % (len(plans), specs[0].paths),
           "interface_nodes": nodes, "grid_nodes": grid_nodes, "steps": steps, "warmup": warmup,
           "path_steps_per_s": path_steps * steps / t, "meshes_per_s": len(plans) * steps / t,
           "ms_per_step": 1000.0 * t / steps, "ms_fill_and_solves": ms_solve,
           "ms_interface_mc": 1000.0 * t / steps - ms_solve,
           "solve_roofline": {"bound": "hbm", "achieved": solve_gbs, "peak": hbm, "unit": "GB/s",
                              "frac": solve_gbs / hbm, "node_iterations": node_its,
                              "bytes_per_node_iteration": SOLVE_BYTES_PER_NODE_ITERATION,
                              "peak_basis": "%s hbm_gbs" % peak_kind,
                              "note": "multigrid-preconditioned FP32 CG: algorithmic bytes of "
                                      "level 0 per interior node and iteration x the nodes and "
                                      "iterations the solves ran, over the fill + solve phase"},
           "precision_bias": bias_on_sample(N, [specs[0], specs[len(specs) // 2]]),
           "jacobi_pcg": {"ms_fill_and_solves": ms_jac, "solve_max_iterations": its_jac,
                          "node_iterations": node_its_jac, "solves_converged": ok_jac,
                          "note": "the same solves with the diagonal preconditioner"},
           "max_stderr": max_se, "solves_converged": solve_ok, "solve_max_iterations": max_iter,
           "path_steps_per_batch": path_steps, "batch_create_s": t_create, "autotune": tuned,
           "gpu_launches": int(launches), "clocks": clocks,
           "l2": "flushed before each timed run"}
    batch.close()
    for p in plans:
        p.close()
    return out


def serve_leg(rates, count, target_stderr, n_max, precision=W.FP32_STEP, max_batch=64,
              reuse_pilot=True, seed=0, ideal=False, **server_kw):
    """Serving runs: a Poisson stream of `count` mesh requests per rate (n
    log-uniform 65..n_max, splits 2..8, 1-3 bumps, dt = 5e-5), paths per node
    from a 1024-path pilot for the std-err target, continuous batching;
    p50/p99 latency and meshes/s per rate.  ideal: also the same requests of
    the last rate, at the paths per node the server chose, as one batch (the
    rate the path kernels reach on these meshes without arrivals or pilots)."""
    import torch
    from paper_1310_3435_gb300 import native as N
    from paper_1310_3435_gb300 import serving as S
    out = []
    res = []
    for rate in rates:
        arr = W.config5(count=count, rate=rate, seed=seed, n_max=n_max)
        reqs = [S.Request(i, W.MeshSpec(**{**a.spec.__dict__, "precision": precision}), a.t)
                for i, a in enumerate(arr)]
        kw = dict(hbm_budget=150e9, n_streams=3, max_batch=max_batch,
                  target_stderr=target_stderr, reuse_pilot=reuse_pilot)
        kw.update(server_kw)
        srv = S.Server(**kw)
        t0 = time.perf_counter()
        res = srv.run(reqs)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        del reqs
        summ = S.summarize(res)
        summ.update({"rate_req_s": rate, "wall_s": wall, "batches_launched": srv.launches,
                     "peak_budget_bytes": srv.peak_used,
                     "device_busy": S.busy_fraction(srv.trace)})
        out.append(summ)
    ideal_line = None
    if ideal and res:
        paths = {r.rid: r.paths for r in res if r.status == "ok"}
        specs = [r.spec for r in sorted(res, key=lambda r: r.rid) if r.rid in paths]
        plans = [N.Plan(sp) for sp in specs]
        chunk = 1024 if reuse_pilot else 0
        mcs = [p.mc_params(paths=paths[r], chunk=chunk)
               for p, r in zip(plans, sorted(paths))]
        stream = torch.cuda.Stream()
        with N.Batch(plans, mcs, [p.solve_params() for p in plans]) as B:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.run(stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1000.0
            steps = sum(int(B.stats(i, allow_not_converged=True)[0].path_steps)
                        for i in range(len(plans)))
        for p in plans:
            p.close()
        ideal_line = {"requests": len(plans), "seconds": sec, "path_steps_per_s": steps / sec,
                      "meshes_per_s": len(plans) / sec,
                      "served_over_ideal": out[-1]["path_steps_per_s"] / (steps / sec),
                      "note": "the last rate's requests at the served paths per node as one "
                              "batch: the rate the kernels reach on these meshes"}
    return {"workload": "Poisson stream, n log-uniform 65..%d, splits 2..8, 1-3 bumps, dt=5e-5, "
                        "std-err target %g (paths per node from a 1024-path pilot%s), %s stepping"
                        % (n_max, target_stderr, ", continued by the final run" if reuse_pilot else "",
                           "FP32" if precision == W.FP32_STEP else "FP64"),
            "requests_per_rate": count, "rates": out, "ideal_batch": ideal_line}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--config", default="config2",
                    choices=["config1", "config2", "config3", "config4"])
    ap.add_argument("--count", type=int, default=256, help="meshes (config3) or requests (--serve)")
    ap.add_argument("--serve", action="store_true", help="serving run (config 5) instead")
    ap.add_argument("--precision-report", action="store_true",
                    help="FP32 stepping vs the FP64 oracle on a node subsample (+ full-N run)")
    ap.add_argument("--sample-nodes", type=int, default=64)
    ap.add_argument("--sample-paths", type=int, default=4096)
    ap.add_argument("--no-full", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--quality-report", action="store_true",
                    help="mesh quality of DD and few-point meshes on the running example")
    ap.add_argument("--quality-dt", type=float, default=1e-4)
    ap.add_argument("--stepper", choices=["euler", "exponential"], default="euler",
                    help="time stepping of the paths (exponential: mean step dt)")
    ap.add_argument("--exit-test", choices=["end", "bridge"], default="end")
    ap.add_argument("--dt", type=float, default=0.0, help="override the workload's (mean) step")
    ap.add_argument("--paper-performance", action="store_true",
                    help="the paper's performance study (five rings, 4x4, n = 37..197)")
    ap.add_argument("--table-tn", type=int, default=0,
                    help="replace the density by a tabulated ln w on this many nodes per side")
    ap.add_argument("--rates", type=float, nargs="+", default=[0.5, 1.0, 2.0])
    ap.add_argument("--n-max", type=int, default=1025)
    ap.add_argument("--target-stderr", type=float, default=1e-3)
    ap.add_argument("--max-batch", type=int, default=64)
    ap.add_argument("--precision", type=int, default=None, help="0 FP64, 1 FP32 stepping")
    ap.add_argument("--ref-budget", type=float, default=15.0,
                    help="seconds of CPU work per oracle sample")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--fp64-paths", type=int, default=2048,
                    help="paths per node of the plain-FP64 GPU comparison leg")
    ap.add_argument("--no-paper-stepper", action="store_true",
                    help="leave the exponential-stepper (lambda = 1e4, bridge) leg out of the line")
    ap.add_argument("--no-batched", action="store_true",
                    help="leave the batched (256 uneven meshes) leg out of the line")
    ap.add_argument("--no-served", action="store_true",
                    help="leave the served legs out of the line")
    ap.add_argument("--served-rates", type=float, nargs="+", default=[4.0, 16.0])
    ap.add_argument("--served-count", type=int, default=200)
    ap.add_argument("--served-stderr", type=float, default=5e-3)
    ap.add_argument("--fp64-served-rate", type=float, default=0.3)
    ap.add_argument("--fp64-served-count", type=int, default=12)
    ap.add_argument("--chunk", type=int, default=0, help="paths per work item (0: automatic)")
    ap.add_argument("--paths", type=int, default=0,
                    help="override paths per node (profiling runs on a small case)")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.serve:
        return run_serve(args)
    if args.precision_report:
        return run_precision(args)
    if args.quality_report:
        return run_quality(args)
    if args.paper_performance:
        return run_paper_performance(args)
    if args.config == "config3":
        return run_batched(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())

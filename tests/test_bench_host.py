"""Host-side logic of bench.py (no GPU): the algorithmic operation counts the
roofline divides by, the guard that keeps a recorded DRAM traffic figure
tied to the kernel source it was measured on, the workload options, and the
reference arm's JSON line (the FP64 oracle timed on the host cores)."""
import argparse
import json

import pytest

import bench
import workloads as W


def _args(**kw):
    base = dict(config="config2", paths=0, dt=0.0, stepper="euler", exit_test="end", table_tn=0,
                gpus=1, steps=1, warmup=0, ref_budget=0.3)
    base.update(kw)
    return argparse.Namespace(**base)


def test_operation_counts():
    # the ring step: Philox 30, uniforms 4, Box-Muller 9, drift 21, update 4,
    # exit test 6, step count and cap 2
    assert bench.OPS_PER_STEP_RING_FP32 == 76
    assert bench.ops_per_step(W.STEP_EULER, W.EXIT_END_OF_STEP) == 76
    assert bench.ops_per_step(W.STEP_EULER, W.EXIT_BRIDGE) == 80.5
    assert bench.ops_per_step(W.STEP_EXPONENTIAL, W.EXIT_END_OF_STEP) == 98
    assert bench.ops_per_step(W.STEP_EXPONENTIAL, W.EXIT_BRIDGE) == 104
    # the tabulated density's drift (17) replaces the ring's (21)
    assert bench.ops_per_step(W.STEP_EULER, W.EXIT_END_OF_STEP, W.FAMILY_TABLE) == 72
    assert bench.ops_per_step(W.STEP_EXPONENTIAL, W.EXIT_BRIDGE, W.FAMILY_TABLE) == 100


def test_traffic_is_reported_only_for_its_workload_and_kernel_source(monkeypatch):
    import hashlib
    import os
    src = os.path.join(bench.ROOT, "paper_1310_3435_gb300", "csrc", "mc.cu")
    with open(src, "rb") as fh:
        current = hashlib.sha256(fh.read()).hexdigest()
    # a figure recorded on the current source is reported for its workload
    monkeypatch.setitem(bench.PATH_KERNEL_TRAFFIC, "source_sha256", current)
    spec = bench.bench_spec(_args())
    assert bench.path_kernel_traffic(spec) == bench.PATH_KERNEL_TRAFFIC["bytes"]
    # another workload, or another kernel source: no figure
    for other in (_args(paths=4096), _args(stepper="exponential"), _args(exit_test="bridge"),
                  _args(table_tn=65), _args(dt=2e-5)):
        assert bench.path_kernel_traffic(bench.bench_spec(other)) is None
    monkeypatch.setitem(bench.PATH_KERNEL_TRAFFIC, "source_sha256", "0" * 64)
    assert bench.path_kernel_traffic(spec) is None


def test_workload_options():
    spec = bench.bench_spec(_args())
    assert (spec.n, spec.sx, spec.sy, spec.family, spec.paths, spec.dt) == \
        (257, 4, 4, W.FAMILY_RING, 100000, 1e-5)
    assert spec.precision == W.FP32_STEP and spec.stepper == W.STEP_EULER
    e = bench.bench_spec(_args(stepper="exponential", exit_test="bridge", dt=1e-4, paths=512))
    assert (e.stepper, e.exit_test, e.dt, e.paths) == (W.STEP_EXPONENTIAL, W.EXIT_BRIDGE, 1e-4, 512)
    assert "exponential steps" in e.label and "bridge" in e.label
    t = bench.bench_spec(_args(table_tn=33))
    assert t.family == W.FAMILY_TABLE and int(t.params[0]) == 33 and len(t.params) == 1 + 33 * 33
    assert bench.bench_spec(_args(), seed=7).seed == 7
    assert bench.bench_spec(_args(config="config4")).n == 1025


def test_reference_arm_line(capsys):
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0",
                       "--ref-budget", "0.3"]) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == "SDE path-steps/s"
    assert line["unit"] == "path-steps/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "path-steps/s",
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith("257x257 4x4 ring")


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(_args()) == 0
    assert capsys.readouterr().out == ""


@pytest.mark.parametrize("steps,seconds", [(10, 2.0), (0, 1.0)])
def test_achieved_rate(steps, seconds):
    assert bench.achieved_steps_per_s(steps, seconds) == pytest.approx(steps / seconds)


def test_further_example_monitors():
    """§4's monitors as the quality report feeds them: the Huang-Sloan ln rho
    table against the printed formula at its nodes (row b is y = b/(tn-1)),
    and the ridge parameters against the Mackenzie front's 1/rho."""
    import math
    tn = 9
    L = bench.huang_sloan_ln_rho(tn)
    assert L.shape == (tn, tn)
    for a, b in ((0, 0), (8, 4), (6, 2), (3, 7)):
        x, y = a / (tn - 1.0), b / (tn - 1.0)
        e = math.exp(15.0 * (x - 1.0))
        rho = math.sqrt(1.0 + 0.7 * (15.0 ** 2 * e ** 2 * math.sin(math.pi * y) ** 2 +
                                     (1.0 - e) ** 2 * math.cos(math.pi * y) ** 2 * math.pi ** 2))
        assert L[b, a] == pytest.approx(math.log(rho), rel=1e-13, abs=1e-15)
    A, k, t0, amp, f = bench.MACKENZIE_RIDGE
    for x, y in ((0.1, 0.6), (0.3, 0.75), (0.8, 0.25)):
        ridge = 1.0 + A * math.exp(-k * (y - t0 - amp * math.sin(2 * math.pi * f * x)) ** 2)
        rho = 1.0 / (1.0 + 10.0 * math.exp(-50.0 * (y - 0.5 - 0.25 * math.sin(2 * math.pi * x)) ** 2))
        assert ridge == pytest.approx(1.0 / rho, rel=1e-14)

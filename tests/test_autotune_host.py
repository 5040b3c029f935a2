"""Autotuner host logic on the CPU with a stand-in timer: bucketing, the
fastest candidate wins, results are cached and reused."""
import workloads as W
from paper_1310_3435_gb300 import autotune as A


def test_picks_fastest_and_caches(tmp_path):
    calls = []

    def timer(kind, spec, value):
        calls.append((kind, value))
        if kind == "mc":
            return {256: 3.0, 1024: 1.0, 4096: 2.0}[value]
        return {256: 5.0, 512: 4.0, 1024: 6.0}[value]

    path = str(tmp_path / "tune.json")
    t = A.Autotuner(timer=timer, device_name="fake", path=path)
    spec = W.config3(count=1, precision=W.FP64)[0]
    got = t.tune(spec)
    assert got == {"chunk": 1024, "block_threads": 512}
    assert len(calls) == 6
    # FP32 stepping keeps the automatic work-item size; only the solve is tuned
    spec32 = W.config3(count=1)[0]
    assert t.tune(spec32) == {"chunk": 0, "block_threads": 512}
    assert len(calls) == 6
    t.save()
    t2 = A.Autotuner(timer=timer, device_name="fake", path=path)
    assert t2.tune(spec) == got
    assert len(calls) == 6                        # cached: no more timing


def test_buckets_separate_different_work():
    small = W.config1()
    big = W.config2()
    assert A.mc_bucket(small, 61) != A.mc_bucket(big, 1521)
    assert A.solve_bucket(small) != A.solve_bucket(big)
    assert A.largest_subdomain(small) == 15 * 15
    assert A.largest_subdomain(big) == 63 * 63


def test_batch_solve_size_is_the_fastest_candidate():
    times = {512: 28.0, 1024: 38.0, 256: 30.0}
    t = A.Autotuner(timer=lambda kind, spec, c: times[c], device_name="fake",
                    path="/nonexistent/autotune.json")
    assert t.tune_batch_solve([], [], [], candidates=(512, 1024)) == 512
    assert t.tune_batch_solve([], [], [], candidates=(1024,)) == 1024


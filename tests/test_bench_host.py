"""Host-side arithmetic of bench.py: the kernel groups read from kg_step_timed, the
algorithmic bytes of the roofline, the double-float operation count and the guard that
drops a stored DRAM-traffic figure once the kernel sources change."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_kernel_groups(bench):
    names, ms = bench.kernel_groups([1.4, 0.65, 2.06, 0.0, 0.0, 0.65])
    assert names == ["x", "yf", "z", "yi"] and ms == [1.4, 0.65, 2.06, 0.65]
    names, ms = bench.kernel_groups([9.3, 3.5, 3.5, 0.94, 3.5, 3.5])
    assert names == ["x", "yf", "zf", "update", "zi", "yi"] and len(ms) == 6


def test_algorithmic_bytes(bench):
    S = 512 * 512 * 257 * 16
    per, step = bench.algorithmic_bytes("df64", 512)
    assert step == 11 * S                                   # 8 W + 3 S with W = S
    assert per["z"] == 5 * S and per["x"] == 2 * S
    assert per["x"] + per["yf"] + per["z"] + per["yi"] == step   # the fused step moves the ideal bytes
    per, step = bench.algorithmic_bytes("mixed", 512)
    assert step == 7 * S and per["z"] == 4 * S              # W = S / 2


def test_double_float_operation_count(bench):
    ops = bench.df64_fp32_ops(512)
    points = 512 * 512 * 257
    assert ops["col"] == points * 218                      # 218 FP32 operations per point and transform
    pairs = 512 * 512 // 2
    assert ops["x"] == pairs * (512 * (16 + 218 + 4 + 2 + 24 + 218) + 257 * 40)
    assert bench.df64_fft_point_ops(512) == 218
    assert bench.df64_step_ops(512) == ops["x"] + 4 * ops["col"]


def test_traffic_guard(bench, monkeypatch):
    if bench.kernel_sources_sha() == bench.TRAFFIC_SOURCES_SHA:
        assert bench.measured_traffic("df64", "z", 512) == bench.TRAFFIC_512[("df64", "z")]
    monkeypatch.setattr(bench, "TRAFFIC_SOURCES_SHA", "0" * 16)
    assert bench.measured_traffic("df64", "z", 512) is None
    monkeypatch.undo()
    assert bench.measured_traffic("df64", "z", 256) is None


def test_step_schedule(bench):
    # the headline: 5 warm-up steps, 20 timed, the energy every 10 levels
    assert bench.step_schedule(5, 20, 10) == [(5, True), (10, True), (5, False)]
    # a region that ends on a multiple of the cadence does not evaluate there
    assert bench.step_schedule(10, 20, 10) == [(10, True), (10, False)]
    assert bench.step_schedule(10, 10, 10) == [(10, False)]
    for start in range(0, 25):
        for steps in range(1, 45):
            sched = bench.step_schedule(start, steps, 10)
            assert sum(k for k, _ in sched) == steps and all(k >= 1 for k, _ in sched)
            level = start
            for k, ev in sched:
                level += k
                assert ev == (level % 10 == 0 and level < start + steps)

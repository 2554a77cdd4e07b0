"""Host logic of the benchmark's clock record (no GPU): the timed loop waits on the sampler, so
its waits must end whether or not nvidia-smi runs, and the summary must read the sampled
clocks and throttle reasons correctly."""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line(sm, smax, hw="Not Active", cap="Not Active"):
    # index, clocks.sm, clocks.max.sm, power.draw, reasons.active, hw_slowdown,
    # hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    return f"0, {sm}, {smax}, 900.0, 0x0, {hw}, Not Active, Not Active, {cap}"


def test_waits_end_without_a_sampler_process():
    clk = bench.ClockSampler(0)  # never entered: no process
    t0 = time.perf_counter()
    clk.wait_running(timeout=5.0)
    clk.wait_samples(3, timeout=5.0)
    assert time.perf_counter() - t0 < 1.0
    assert clk.summary() == dict(sm_mhz=None, sm_max_mhz=None, reasons=["unsampled"], samples=0)


def test_waits_end_at_their_timeout_when_no_sample_arrives():
    clk = bench.ClockSampler(0)
    clk.proc = object()  # a process that prints nothing
    t0 = time.perf_counter()
    clk.wait_samples(1, timeout=0.2)
    assert 0.15 < time.perf_counter() - t0 < 2.0


def test_summary_reads_clocks_and_reasons():
    clk = bench.ClockSampler(0)
    clk.lines = [_line(2070, 2070), _line(1980, 2070, cap="Active"), _line(2070, 2070), "garbage", ""]
    s = clk.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    clk.lines = [_line(1200, 2070, hw="Active")]
    assert clk.summary()["reasons"] == ["hw_slowdown"]

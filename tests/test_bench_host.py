"""Host logic of bench.py that needs no GPU: the clock record of the timed region
and the count of kernel launches it claims."""
import pytest

import bench


def test_clock_summary_median_under_load_and_reasons():
    # index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    lines = [
        "0, 1980, 2070, 150.2, 0x0, Not Active, Not Active, Not Active, Not Active\n",   # idle: not under load
        "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active\n",
        "0, 2010, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active\n",
        "0, 2040, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active\n",
        "garbage line\n",
        "0, [N/A], 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active\n",  # unreadable: skipped
    ]
    s = bench.summarize_clocks(lines)
    assert s["samples"] == 4
    assert s["sm_mhz"] == 2040.0            # median of the three loaded samples
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert s["power_w_max"] == pytest.approx(1390.5)


def test_clock_summary_reports_every_throttle_reason():
    lines = ["0, 1500, 2070, 800, 0x8, Active, Not Active, Active, Not Active\n",
             "0, 1600, 2070, 820, 0x0, Not Active, Active, Not Active, Not Active\n"]
    s = bench.summarize_clocks(lines)
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert s["sm_mhz"] == 1550.0
    assert bench.summarize_clocks(["", "x, y\n"]) is None


def test_launch_count_of_one_iteration():
    # 1024 detectors in one chunk: map copy in and out, forward and filter, one
    # inverse + binning launch over four 256-detector partial maps and its flush
    # (A: 6), the CG update (6) and the circulant apply (7)
    assert bench.launches_per_iteration(1024, 1024) == 6 + 6 + 7
    # two chunks of 512: each forward, filter, one inverse + binning, one flush
    assert bench.launches_per_iteration(1024, 512) == 2 + 2 * 4 + 6 + 7
    # 4096 detectors in one chunk: eight partial maps per inverse launch, two launches
    assert bench.launches_per_iteration(4096, 4096) == 2 + 2 + 2 * 2 + 6 + 7
    # a ragged last chunk of 100 detectors still takes its own launches
    assert bench.launches_per_iteration(612, 256) == 2 + 3 * 4 + 6 + 7


def test_oracle_solve_estimate():
    est = bench.oracle_solve_estimate(2.0e8, 1 << 30, {"circulant": {"iterations": 434}, "binned": {}})
    assert est["value"] == pytest.approx((1 << 30) / 2.0e8 * 434)
    assert est["iterations"] == 434 and "estimate" in est["what"]
    assert bench.oracle_solve_estimate(2.0e8, 1 << 30, None) is None
    assert bench.oracle_solve_estimate(2.0e8, 1 << 30, {"binned": {"iterations": 3}}) is None

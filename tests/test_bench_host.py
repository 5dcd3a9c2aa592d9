"""Host logic of bench.py on CPU: the clock record taken during the timed region and the RCS error
metric that gates the fast path."""
import math

import numpy as np

import bench


def _line(sm, smax, hw="Not Active", thermal="Not Active", sw_thermal="Not Active", power="Not Active"):
    # index, clocks.sm, clocks.max.sm, power.draw, active reasons, hw, hw thermal, sw thermal, sw power
    return f"0, {sm}, {smax}, 700.0, 0x0, {hw}, {thermal}, {sw_thermal}, {power}\n"


def test_clock_summary_keeps_samples_inside_the_timed_region():
    lines = [_line(1000, 2070), _line(1100, 2070), _line(2070, 2070), _line(2055, 2070), _line(2040, 2070)]
    out = bench.ClockSampler.summarise(lines, 2)
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2055.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == []


def test_clock_summary_falls_back_to_the_last_sample_before_a_short_region():
    lines = [_line(1500, 2070), _line(2070, 2070)]
    out = bench.ClockSampler.summarise(lines, 2)
    assert out["samples"] == 0
    assert out["sm_mhz"] == 2070.0


def test_clock_summary_reports_slowdown_reasons():
    lines = [_line(2070, 2070), _line(1800, 2070, thermal="Active"), _line(1900, 2070, power="Active"),
             "garbage line\n"]
    out = bench.ClockSampler.summarise(lines, 0)
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert out["sm_mhz"] == 1900.0


def test_rcs_db_error_known_offsets_and_null_floor():
    ref = np.array([1.0, 0.5, 1e-5, 0.25])
    s = ref * np.array([10 ** (0.05 / 10), 10 ** (-0.02 / 10), 100.0, 1.0])
    # the deep null (45 dB below the maximum) is outside the 30 dB floor
    assert math.isclose(bench.rcs_db_error(s, ref), 0.05, rel_tol=1e-9)
    assert math.isclose(bench.rcs_db_error(s, ref, floor_db=60.0), 20.0, rel_tol=1e-9)

"""bench.py's summary of the nvidia-smi samples taken during the timed region:
the median SM clock, the largest maximum, every throttle reason seen Active
(a run showing hw_slowdown, hw_thermal_slowdown or sw_thermal_slowdown is
rejected, sw_power_cap is kept and noted), and lines that do not parse
(a header, N/A fields, a truncated last line) skipped."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"{sm}, {mx}, 850.12, {hw}, {hwt}, {swt}, {cap}"


def test_clean_samples():
    lines = [_line(2070, 2070)] * 4 + [_line(2055, 2070)]
    s = bench.summarise_clocks(lines)
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 5}


def test_reasons_collected_and_median():
    lines = [_line(1980, 2070, cap="Active"), _line(2070, 2070), _line(1500, 2070, hwt="Active"),
             _line(2010, 2070, swt="Active"), _line(2070, 2070, hw="Active")]
    s = bench.summarise_clocks(lines)
    assert s["sm_mhz"] == 2010.0
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert s["samples"] == 5


def test_unparsable_lines_skipped():
    lines = ["clocks.sm [MHz], clocks.max.sm [MHz], power.draw [W], a, b, c, d",  # a header
             "[N/A], 2070, 800.0, Not Active, Not Active, Not Active, Not Active",
             "2070, 2070, 8",  # truncated
             _line(2040, 2070)]
    s = bench.summarise_clocks(lines)
    assert s == {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 1}


def test_no_samples():
    assert bench.summarise_clocks([]) is None
    assert bench.summarise_clocks(["garbage"]) is None

"""Host logic of the bench that needs no GPU: the clock record taken during the timed region
(median SM clock under load, the highest max clock, and every throttle reason seen)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def sampler(rows):
    c = bench.ClockSampler(0)
    c.samples = [[x.strip() for x in r.split(",")] for r in rows]
    return c.summary()


def test_clock_summary_without_throttling():
    s = sampler(["2070, 2070, 900.5, Not Active, Not Active, Not Active, Not Active",
                 "2055, 2070, 1100.0, Not Active, Not Active, Not Active, Not Active",
                 "2070, 2070, 1200.0, Not Active, Not Active, Not Active, Not Active"])
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}


def test_clock_summary_reports_every_reason_seen():
    s = sampler(["1800, 2070, 1400.0, Not Active, Not Active, Not Active, Active",
                 "1500, 2070, 1390.0, Active, Not Active, Active, Not Active",
                 "[N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]"])
    assert s["sm_mhz"] == 1650.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    assert sampler([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}

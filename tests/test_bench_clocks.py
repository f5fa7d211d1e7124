"""bench.py's clock record without a GPU: the summary keeps only the samples
taken after the sampler's first line (the timed region), takes their median
SM clock and lists every throttle reason seen active among them."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

NA = "Not Active"


def _line(sm, mx=2070, reasons=(NA, NA, NA, NA)):
    return ", ".join([str(sm), str(mx), "900.0", "0x0", *reasons])


def test_summary_keeps_samples_after_the_first():
    c = bench.Clocks(0)
    c.lines = [_line(345), _line(2070), _line(2055), _line(2070, reasons=(NA, NA, NA, "Active"))]
    c.first = 1                     # the idle sample taken before the timed region
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_summary_reports_throttle_reasons_and_skips_bad_lines():
    c = bench.Clocks(0)
    c.lines = ["garbage", _line(1800, reasons=("Active", NA, "Active", NA)), "[N/A], 2070, 1, 0, a, b, c, d"]
    s = c.summary()
    assert s["samples"] == 1 and s["sm_mhz"] == 1800.0
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_summary_falls_back_to_the_last_sample():
    c = bench.Clocks(0)
    c.lines = [_line(2070)]
    c.first = 1                     # the timed region was shorter than one sampling interval
    assert c.summary()["samples"] == 1
    assert bench.Clocks(0).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}

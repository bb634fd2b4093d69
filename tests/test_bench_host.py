"""Host-side pieces of the benchmark (no GPU): the clock record taken during a
timed region, and the peaks its roofline fractions divide by."""
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


def test_clock_summary_reports_median_and_reasons(bench):
    c = bench.ClockSampler(0)
    # rows as nvidia-smi prints them: clocks.sm, clocks.max.sm, power, hw, hw thermal, sw thermal, sw power cap
    c.rows = [["2070", "2070", "900.1", "Not Active", "Not Active", "Not Active", "Not Active"],
              ["1995", "2070", "1390.0", "Not Active", "Not Active", "Not Active", "Active"],
              ["2070", "2070", "1200.0", "Not Active", "Not Active", "Not Active", "Not Active"]]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.rows[0][4] = "Active"          # a thermal slowdown anywhere in the region is reported
    assert "hw_thermal_slowdown" in c.summary()["reasons"]
    c.rows = []
    assert c.summary()["reasons"] == ["unsampled"]


def test_roofline_peaks(bench):
    assert bench.sfu_ex2_per_clk_sm() == pytest.approx(31.96, abs=0.05)   # the committed probe table
    p = bench.measured_peaks()
    assert p["source"] in ("measured", "fallback")
    assert p["bf16_tflops_sustained"] > 0 and p["hbm_gbs"] > 0
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert p["source"] == "measured"

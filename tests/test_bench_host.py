"""Host-side logic of bench.py that needs no GPU: the clock-sample summary
(median SM clock, max clock, throttle reasons) that decides whether a timed
run is kept, and the measured-peaks file it divides by."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def sampler(lines):
    c = bench.ClockSampler(0)
    c.lines = list(lines)
    return c


def test_clock_summary_median_max_and_reasons():
    lines = [
        "2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "1980, 2070, 1400.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "[N/A], 2070, 10.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = sampler(lines).summary()
    assert s == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3}


def test_clock_summary_reports_every_slowdown_kind():
    lines = ["1500, 2070, 1000, 0x8, Active, Not Active, Not Active, Not Active",
             "1400, 2070, 1000, 0x8, Not Active, Active, Not Active, Not Active",
             "1300, 2070, 1000, 0x8, Not Active, Not Active, Active, Not Active"]
    s = sampler(lines).summary()
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert s["sm_mhz"] == 1400.0


def test_clock_summary_without_samples_is_none():
    assert sampler([]).summary() is None
    assert sampler(["", "a, b"]).summary() is None


def test_measured_peaks_file_is_read():
    pk = bench.peaks()
    if os.path.exists(bench.PEAKS_FILE):
        assert pk.get("hbm_gbs", 0) > 1000 and pk.get("bf16_tflops", 0) > 100
    else:
        assert pk == {}


def test_stencil_roofline_traffic_only_for_the_captured_grid_and_shape():
    """The ncu DRAM bytes are reported only for the grid and thread shape they
    were captured on; achieved = 12 Nd Ns bytes / the median launch time."""
    nd, ns = bench.RING_CAPTURED_ND, 1300
    stage = [{"stencil_launches": 20, "stencil_ms": 20 * 5.0, "nonlocal_ms": 20 * 1.0}]
    pk = {"hbm_gbs": 6000.0}
    r = bench.stencil_roofline(stage, nd, ns, "mixed", pk, None,
                               {"shape": bench.RING32_CAPTURED_SHAPE})
    assert abs(r["achieved"] - 12 * nd * ns / 5e-3 / 1e9) < 1e-6 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / 6000.0) < 1e-12
    assert abs(r["traffic"] - bench.RING32_DRAM_BYTES_PER_ORBITAL * ns) < 1.0
    other = bench.stencil_roofline(stage, nd, ns, "mixed", pk, None,
                                   {"shape": bench.RING32_CAPTURED_SHAPE + 3})
    assert other["traffic"] is None and other["achieved"] == r["achieved"]
    slab = bench.stencil_roofline(stage, 64 * 64 * 160, ns, "mixed", pk, None,
                                  {"shape": bench.RING32_CAPTURED_SHAPE})
    assert slab["traffic"] is None
    assert bench.stencil_roofline(stage, nd, ns, "mixed", pk, None)["traffic"] is None

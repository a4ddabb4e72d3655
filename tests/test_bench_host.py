"""Host-side arithmetic of the benchmark, on the CPU: the Eq. 11 filter's
tap count behind its FLOP roofline, the clock record's summary of
nvidia-smi samples, and the rounding of the line's closing summary."""
import numpy as np
import pytest

import bench


@pytest.mark.parametrize("H,W,r", [(1, 1, 0), (5, 7, 1), (9, 4, 3), (3, 3, 5), (16, 11, 8), (2, 30, 4)])
def test_denoise_taps_counts_every_window_pair_inside_the_image(H, W, r):
    ys, xs = np.mgrid[0:H, 0:W]
    brute = 0
    for y, x in zip(ys.ravel(), xs.ravel()):
        brute += int(np.sum((np.abs(ys - y) <= r) & (np.abs(xs - x) <= r)))
    assert bench.denoise_taps(H, W, r) == brute


def test_clock_summary_reads_nvidia_smi_samples():
    s = bench.ClockSampler(None)
    s.lines = [
        "2070, 2070, 900.5, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 1100.0, Not Active, Not Active, Not Active, Active",
        "1980, 2070, 1390.2, Not Active, Not Active, Not Active, Active",
        "[N/A], 2070, 10.0, Not Active, Not Active, Not Active, Not Active",  # unreadable sample: skipped
        "2070, 2070",                                                          # truncated line: skipped
    ]
    out = s.summary()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2055.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    s.lines = ["1500, 2070, 700, Active, Not Active, Active, Not Active"]
    assert s.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    s.lines = []
    assert s.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}


def test_summary_figures_are_rounded_and_absent_entries_dropped():
    x = {"forward": 3029.4567, "fwd_bwd": {"value": 1890.123456, "unfused": None}, "p99": [124.56789, 2],
         "name": "corner"}
    assert bench.short_figures(x) == {"forward": 3029.0, "fwd_bwd": {"value": 1890.0}, "p99": [124.6, 2],
                                      "name": "corner"}

"""Host-side arithmetic of bench.py, on CPU: the clock summary that decides whether a timed
region is kept (median SM clock, throttle reasons seen while timing), the per-class roofline
fractions (algorithmic bytes over CUDA-event time against the measured and nominal HBM
peaks, and FP64 flops against the derived FP64 peak), the derived FP64 peak itself, and the
peaks file."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
bench = pytest.importorskip("bench")


def _sample(mhz, mx=2070, active="0x0", hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return [str(mhz), str(mx), active, hw, hwt, swt, cap]


def test_clock_summary_median_and_reasons():
    cs = bench.ClockSampler("0")
    cs.samples = [_sample(2070), _sample(1980, cap="Active"), _sample(2070), _sample(1500, hwt="Active"),
                  ["[N/A]", "2070", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]]
    s = cs.summary()
    assert s["samples"] == 4                      # the unparsable line is skipped
    assert s["sm_mhz"] == pytest.approx(2025.0)   # median of 1500, 1980, 2070, 2070
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_summary_clean_and_empty():
    cs = bench.ClockSampler("0")
    cs.samples = [_sample(2070) for _ in range(5)]
    assert cs.summary() == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 5}
    empty = bench.ClockSampler("0").summary()
    assert empty["sm_mhz"] is None and empty["samples"] == 0 and empty["reasons"] == []


def test_fp64_peak_is_the_unit_count_times_the_clock():
    # 152 SMs x 2 FP64 FMA per clock x 2 flops per FMA x 2070 MHz
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(152 * 2 * 2 * 2.070e9 / 1e12)
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(1.25856)


def test_class_rooflines_fractions():
    # 1 GB in 1 ms = 1000 GB/s; 2e9 flops in 1 ms = 2 TFLOP/s
    prof64 = {"bicg_v": {"launches": 4, "ms": 1.0, "bytes": 1e9, "flops": 2e9},
              "proj_update": {"launches": 1, "ms": 0.0, "bytes": 1e9, "flops": 1e9}}
    prof32 = {"bicg_x": {"launches": 2, "ms": 2.0, "bytes": 8e9, "flops": 0.0}}
    out = bench.class_rooflines(prof64, prof32, 5000.0)
    v = out["stencil.bicg_v.f64"]
    assert v["us_per_launch"] == 250.0
    assert v["gbs"] == 1000.0
    assert v["hbm_frac"] == pytest.approx(0.2)
    assert v["hbm_frac_nominal"] == pytest.approx(1000.0 / bench.NOMINAL_HBM_GBS)
    assert v["fp64_tflops"] == pytest.approx(2.0)
    assert v["fp64_frac"] == pytest.approx(round(2.0 / bench.FP64_PEAK_TFLOPS, 4))
    assert "projection.proj_update.f64" not in out          # no time recorded: no entry
    x = out["bicgstab_update.bicg_x.f32"]
    assert x["gbs"] == 4000.0 and x["hbm_frac"] == pytest.approx(0.8)
    assert "fp64_tflops" not in x


def test_measured_peaks_file():
    peaks, src = bench.measured_peaks()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert src == "measured"
        assert peaks["hbm_gbs"] > 1000.0
    else:
        assert src == "fallback" and peaks["hbm_gbs"] == 6800.0


def test_weak_scaling_rate_counts_every_rank():
    # 3 units per rank on 4 ranks in 1500 ms (the slowest rank's time): 8 units/s
    assert bench.weak_scaling_rate(3, 1500.0, 4) == pytest.approx(8.0)

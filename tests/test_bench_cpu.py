"""The benchmark's byte accounting and roofline arithmetic, on the CPU.

The fused path must move n·P·2 bytes of raw frames, P·12 of masters and P·8
of outputs per set (2 + 20/n bytes per raw pixel); the roofline divides such
algorithmic bytes by the dominant kernel's event-timed duration, and the
issue roofline divides its ncu instruction count by the same duration.
"""
import pytest

import bench


def test_algorithmic_bytes_per_raw_pixel():
    P = 4096 * 4096
    # deep: 32 frames of 4096^2, bilinear, fused: P (2n + 20)
    assert bench.algorithmic_bytes("reduce", [(4096, 4096, 32)], "bilinear") == P * (64 + 20)
    # bands: spline prefilter reads raw and masters and writes coefficients,
    # the reduction reads 4 B per sample and writes the outputs
    P1 = 1024 * 1024
    bands = [(1024, 1024, 10)] * 3
    assert bench.algorithmic_bytes("prefilter", bands, "spline3") == 3 * (10 * P1 * 6 + P1 * 12)
    assert bench.algorithmic_bytes("reduce", bands, "spline3") == 3 * (10 * P1 * 4 + P1 * 8)
    # a deep spline band (180 frames) combines from 4 B per sample
    P2 = 1020 * 1020
    assert bench.algorithmic_bytes("combine", [(1020, 1020, 180)], "spline3") == P2 * (720 + 8)
    assert set(bench.step_bytes([(1020, 1020, 180)], "spline3")) == {"reduce", "prefilter",
                                                                     "combine"}


def test_roofline_of_the_deep_workload():
    shapes = [(4096, 4096, 32)]
    by = bench.step_bytes(shapes, "bilinear")
    steps, ms = 10, 2.09
    prof = {"reduce": (ms * steps, steps), "prefilter": (0.0, 0)}
    rf = bench.roofline(prof, steps, by, ms, by["reduce"], "deep", sm_count=152)
    peak, _ = bench.measured_peaks()
    assert rf["kernel"] == "reduce" and rf["bound"] == "hbm"
    assert rf["achieved"] == pytest.approx(by["reduce"] / (ms * 1e-3) / 1e9, rel=1e-3)
    assert rf["frac"] == pytest.approx(rf["achieved"] / peak, rel=1e-3)
    assert rf["traffic"] == bench.TRAFFIC["deep"][2]
    # 1.292 G warp instructions in 2.09 ms against 152 x 4 x 2.07 GHz
    iss = rf["issue"]
    assert iss["peak"] == pytest.approx(152 * 4 * bench.sm_max_mhz() / 1e3, rel=1e-3)
    assert iss["frac"] == pytest.approx(1_292_075_776 / 2.09e-3 / (iss["peak"] * 1e9), rel=1e-3)


def test_roofline_reports_no_counters_for_changed_sources(monkeypatch):
    shapes = [(1024, 1024, 10)] * 3
    by = bench.step_bytes(shapes, "spline3")
    prof = {"prefilter": (1.4, 10), "reduce": (0.9, 10)}
    rf = bench.roofline(prof, 10, by, 0.235, by["reduce"], "bands", sm_count=152)
    assert rf["kernel"] == "prefilter" and rf["traffic"] is not None and rf["issue"] is not None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    rf = bench.roofline(prof, 10, by, 0.235, by["reduce"], "bands", sm_count=152)
    assert rf["traffic"] is None and rf["issue"] is None
    # workloads without a capture, or without a device, carry none either
    rf = bench.roofline(prof, 10, by, 0.235, by["reduce"], "small", sm_count=152)
    assert rf["traffic"] is None and rf["issue"] is None


def test_sampled_errors_report_the_relative_difference_ranges():
    import numpy as np

    import oracle
    from paper_2008_11486_gb300 import synth
    fs = synth.make_set(48, 40, 6, 3.0, 77, n_stars=10, n_cr=3)
    full = oracle.reduce_set(fs, interp="bilinear")
    # the oracle's own result, rounded to FP32 and scaled by (1 + 1e-6)
    mean = (full["mean"] * (1 + 1e-6)).astype(np.float32)
    med = full["median"].astype(np.float32)
    res = bench.sampled_errors(fs, {"scaled": (mean, med)}, "bilinear", npix=500)
    r = res["scaled"]
    lo90, hi90 = r["mean_dI_90"]
    lo95, hi95 = r["mean_dI_95"]
    assert lo95 <= lo90 <= hi90 <= hi95
    # dI is 1e-6 up to the FP32 rounding of the outputs (about 6e-8)
    assert abs(lo95 - 1e-6) < 1e-7 and abs(hi95 - 1e-6) < 1e-7
    assert r["median_max_rel"] < 1e-7 and res["pixels"] > 400

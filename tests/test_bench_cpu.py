"""The benchmark's byte accounting and roofline arithmetic, on the CPU.

The fused path must move n·P·2 bytes of raw frames, P·12 of masters and P·8
of outputs per set (2 + 20/n bytes per raw pixel); the roofline divides these
algorithmic bytes by the dominant kernel's event-timed duration (and by the
whole step's for ``path_frac``), and the issue roofline divides its ncu
instruction count by the same duration.
"""
import pytest

import bench


def test_path_bytes_per_raw_pixel():
    P = 4096 * 4096
    # deep: 32 frames of 4096^2: P (2n + 20), whatever the interpolation
    assert bench.path_bytes([(4096, 4096, 32)]) == P * (64 + 20)
    # bands: three sets of 10 frames of 1024^2
    P1 = 1024 * 1024
    assert bench.path_bytes([(1024, 1024, 10)] * 3) == 3 * P1 * 40
    # the paper's band of 180 frames: 2 + 20/180 bytes per raw pixel
    P2 = 1020 * 1020
    assert bench.path_bytes([(1020, 1020, 180)]) == P2 * 380
    # the kept count adds 2 bytes per output pixel
    assert bench.path_bytes([(64, 32, 5)], want_nkept=True) == 64 * 32 * 32


def test_roofline_of_the_deep_workload():
    shapes = [(4096, 4096, 32)]
    pb = bench.path_bytes(shapes)
    steps, ms = 10, 2.09
    prof = {"reduce": (ms * steps, steps), "prefilter": (0.0, 0)}
    rf = bench.roofline(prof, steps, pb, ms, "deep", sm_count=152)
    peak, _ = bench.measured_peaks()
    assert rf["kernel"] == "reduce" and rf["bound"] == "hbm"
    assert rf["achieved"] == pytest.approx(pb / (ms * 1e-3) / 1e9, rel=1e-3)
    assert rf["frac"] == pytest.approx(rf["achieved"] / peak, rel=1e-3)
    assert rf["algorithmic_bytes"] == pb
    assert rf["path_frac"] == pytest.approx(rf["frac"], rel=1e-3)  # one kernel: the whole path


def test_roofline_of_a_multi_kernel_step_uses_the_path_bytes():
    """The spline bands: the prefilter dominates; its fraction is the path's
    algorithmic bytes over its own time, and the whole step's fraction is the
    same bytes over the step time."""
    shapes = [(1024, 1024, 10)] * 3
    pb = bench.path_bytes(shapes)
    prof = {"prefilter": (1.415, 10), "reduce": (0.9, 10)}
    rf = bench.roofline(prof, 10, pb, 0.2407, "bands", sm_count=152)
    peak, _ = bench.measured_peaks()
    assert rf["kernel"] == "prefilter"
    assert rf["achieved"] == pytest.approx(pb / 0.1415e-3 / 1e9, rel=1e-3)
    assert rf["path_frac"] == pytest.approx(pb / 0.2407e-3 / 1e9 / peak, rel=1e-3)
    assert rf["kernel_ms"] == {"prefilter": 0.1415, "reduce": 0.09}


def test_roofline_reports_no_counters_for_changed_sources(monkeypatch):
    shapes = [(4096, 4096, 32)]
    pb = bench.path_bytes(shapes)
    prof = {"reduce": (20.9, 10)}
    monkeypatch.setitem(bench.TRAFFIC, "deep", (bench.kernel_source_hash(), "reduce", 123))
    monkeypatch.setitem(bench.ISSUE, "deep", (bench.kernel_source_hash(), "reduce", 456))
    rf = bench.roofline(prof, 10, pb, 2.09, "deep", sm_count=152)
    assert rf["traffic"] == 123 and rf["issue"]["warp_instructions"] == 456
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    rf = bench.roofline(prof, 10, pb, 2.09, "deep", sm_count=152)
    assert rf["traffic"] is None and rf["issue"] is None
    # workloads without a capture, or without a device, carry none either
    rf = bench.roofline(prof, 10, pb, 2.09, "small", sm_count=152)
    assert rf["traffic"] is None and rf["issue"] is None


def test_issue_roofline_arithmetic(monkeypatch):
    monkeypatch.setitem(bench.ISSUE, "deep", (bench.kernel_source_hash(), "reduce",
                                              1_292_075_776))
    iss = bench.issue_roofline("deep", "reduce", 2.09, 152, bench.sm_max_mhz())
    assert iss["peak"] == pytest.approx(152 * 4 * bench.sm_max_mhz() / 1e3, rel=1e-3)
    assert iss["frac"] == pytest.approx(1_292_075_776 / 2.09e-3 / (iss["peak"] * 1e9), rel=1e-3)


def test_cpu_model_is_named():
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()


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

"""Parity of the CUDA path with the FP64 oracle (needs a GPU: -m gpu).

Every case runs the C ABI through the ctypes binding on seeded synthetic
frame sets and compares element by element with the oracle on the same
inputs, at sizes that span several tiles and ragged tile tails."""
import ctypes
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2008_11486_gb300 import build as irp_build
from paper_2008_11486_gb300 import core, synth
from parity_util import compare, gate_e2e, mean_tolerance, sample_tolerance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _native():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    irp_build.build()


def run_fused(fs_list, interp, *, kappa=3.0, max_iter=3, persistent=False, want_stack=True,
              normalize_flat=False, center="mean", ddof=0, onchip=False):
    sets = [core.device_set(fs).alloc_outputs(want_stack=want_stack) for fs in fs_list]
    params = core.reduce_params(interp, core.clip_params(kappa, max_iter, center, ddof),
                                normalize_flat, persistent, spline_onchip=onchip)
    ws = core.reduce_sets(sets, params)
    assert core.sync_status(ws) == 0
    out = []
    for s in sets:
        d = dict(mean=s.mean.cpu().numpy(), median=s.median.cpu().numpy(),
                 nkept=s.nkept.cpu().numpy().astype(np.int32))
        if want_stack:
            d["stack"] = s.stack.cpu().numpy()
        out.append(d)
    return out


def check_against_oracle(fs, got, interp, kappa, max_iter, normalize_flat=False, check_stack=True):
    ref = oracle.reduce_set(fs, interp=interp, kappa=kappa, max_iter=max_iter,
                            normalize_flat=normalize_flat, want_stack=True)
    stats = {}
    st = got["stack"]
    gvalid = ~np.isnan(st)
    # validity of every sample is integer logic: bit-exact
    assert np.array_equal(gvalid, ref["valid"]), "sample validity differs"
    tol = sample_tolerance(fs, interp, oracle)
    if normalize_flat:  # the normalised samples are larger by the flat's mean
        tol = tol * max(1.0, float(np.mean(fs.flat, dtype=np.float64)))
    if check_stack:
        stats["stack"] = compare("stack", st, np.where(ref["valid"], ref["stack"], np.nan), tol)
    # combine on identical inputs: the oracle fed with the GPU's FP32 samples
    same = oracle.combine_stack(np.where(gvalid, st, 0.0), gvalid, kappa=kappa,
                                max_iter=max_iter)
    med_ref = same["median"].astype(np.float32)
    assert np.array_equal(np.isnan(got["median"]), np.isnan(med_ref))
    fin = ~np.isnan(med_ref)
    assert np.array_equal(got["median"][fin].view(np.uint32), med_ref[fin].view(np.uint32)), \
        "median not bit-exact on identical inputs"
    exempt = same["margin"] < 1e-5
    assert exempt.mean() < 1e-3
    kept_ok = (got["nkept"] == same["nkept"]) | exempt
    assert kept_ok.all(), f"clip masks differ at {np.sum(~kept_ok)} non-exempt pixels"
    agree = (got["nkept"] == same["nkept"])
    stats["mean_same_inputs"] = compare("mean(same inputs)", got["mean"], same["mean"],
                                        mean_tolerance(same["mean"]), agree)
    # end to end against the oracle's own FP64 samples: clip results agree
    # except within rounding reach of a threshold; mean and median within the
    # plain tolerance where the measured sample errors allow it
    samp = np.max(np.where(ref["valid"], tol, 0.0), axis=0)
    meas = np.max(np.where(ref["valid"], np.abs(np.where(gvalid, st, 0.0) - ref["stack"]), 0.0),
                  axis=0)
    stats["e2e"] = gate_e2e("e2e", got, ref, samp, kappa, meas=meas)
    return stats


@pytest.mark.parametrize("interp,onchip", [("nearest", False), ("bilinear", False),
                                           ("spline3", False), ("spline3", True),
                                           ("cubic", False)])
def test_fused_small_ragged(interp, onchip):
    fs = synth.make_set(100, 70, 12, 5.0, 501, n_stars=40, n_cr=8)
    got = run_fused([fs], interp, kappa=2.5, onchip=onchip)[0]
    stats = check_against_oracle(fs, got, interp, 2.5, 3)
    print(interp, onchip, stats)


@pytest.mark.parametrize("n", [48, 64])
def test_fused_spline_above_40_frames_both_tile_heights(n):
    """Filtered-row spline sets of 41 to 64 frames: one row per warp (the
    default) and two rows (the other choice) agree bit for bit and with the
    oracle."""
    fs = synth.make_set(90, 60, n, 5.0, 6400 + n, n_stars=25, n_cr=8)
    outs = []
    for rpw in (0, 2):
        s = core.device_set(fs).alloc_outputs(want_stack=False)
        ws = core.reduce_sets([s], core.reduce_params("spline3", core.clip_params(2.5, 3),
                                                      rows_per_warp=rpw))
        assert core.sync_status(ws) == 0
        outs.append(dict(mean=s.mean.cpu().numpy(), median=s.median.cpu().numpy(),
                         nkept=s.nkept.cpu().numpy().astype(np.int32)))
    for k in ("mean", "median", "nkept"):
        assert np.array_equal(outs[0][k].view(np.uint32), outs[1][k].view(np.uint32)), k
    got = run_fused([fs], "spline3", kappa=2.5)[0]
    print(check_against_oracle(fs, got, "spline3", 2.5, 3))
    for k in ("mean", "median"):
        assert np.array_equal(got[k].view(np.uint32), outs[0][k].view(np.uint32)), k


def test_fused_small_config_full_size():
    """5 frames of 512x512, offsets +-5 px, bilinear, 3-sigma 3 iterations."""
    fs = synth.workload_small()
    got = run_fused([fs], "bilinear")[0]
    print(check_against_oracle(fs, got, "bilinear", 3.0, 3))


@pytest.mark.parametrize("onchip", [False, True])
def test_fused_spline_band_full_size_sampled(onchip):
    """One band of the multi-band workload: 10 frames of 1024^2, +-10 px,
    spline (column pass and vertical taps, or the on-chip tile kernel); the
    oracle evaluates sampled pixels (and every edge pixel)."""
    fs = synth.workload_bands(n=10)[0]
    got = run_fused([fs], "spline3", want_stack=False, onchip=onchip)[0]
    rng = np.random.default_rng(7)
    H, W = fs.H, fs.W
    xs = np.concatenate([rng.integers(0, W, 3000), np.arange(W), np.arange(W),
                         np.zeros(H, int), np.full(H, W - 1)])
    ys = np.concatenate([rng.integers(0, H, 3000), np.zeros(W, int), np.full(W, H - 1),
                         np.arange(H), np.arange(H)])
    ref = oracle.reduce_set(fs, interp="spline3", pixels=(xs, ys))
    g = {k: got[k][ys, xs] for k in ("mean", "median", "nkept")}
    samp = sample_tolerance(fs, "spline3", oracle).max(axis=0)[ys, xs]
    print(gate_e2e("spline band", g, ref, samp, 3.0))


def test_persistent_and_batch_invariance():
    """Each set's output is bit-identical alone (plain launch) and inside a
    persistent batch of uneven sets."""
    shapes = [(3, 70, 50), (9, 64, 96), (17, 40, 33), (33, 48, 64), (5, 20, 130)]
    fss = [synth.make_set(W, H, n, 4.0, 900 + i, n_stars=20, n_cr=4)
           for i, (n, W, H) in enumerate(shapes)]
    alone = [run_fused([fs], "bilinear", kappa=2.5, want_stack=False)[0] for fs in fss]
    batch = run_fused(fss, "bilinear", kappa=2.5, persistent=True, want_stack=False)
    for a, b in zip(alone, batch):
        for key in ("mean", "median", "nkept"):
            assert np.array_equal(a[key].view(np.uint8), b[key].view(np.uint8)), key
    # and the batch matches the oracle
    for fs, b in zip(fss, batch):
        ref = oracle.reduce_set(fs, interp="bilinear", kappa=2.5)
        samp = sample_tolerance(fs, "bilinear", oracle).max(axis=0)
        gate_e2e("batch", b, ref, samp, 2.5)


def test_batch_mixing_master_window_forms():
    """Sets of one frame-count bucket (33 to 40 frames) whose master windows
    take different forms share one launch: a premerged window (one exposure
    time, no mask; staged at 12 B a pixel, the largest offsets), a masked set
    and a set of several exposure times (16 B a pixel).  Each set's outputs
    equal its reduction alone bit for bit, in plain and persistent launches,
    and the unmasked ones match the oracle."""
    fa = synth.make_set(90, 70, 36, 9.0, 7301, n_stars=20, n_cr=6)
    fb = synth.make_set(90, 70, 38, 3.0, 7302, n_stars=20, n_cr=6)
    fc = synth.make_set(90, 70, 40, 3.0, 7303, n_stars=20, n_cr=6)
    fc.exptime = np.linspace(30.0, 90.0, 40).astype(np.float32)
    mask = (np.random.default_rng(7).random((70, 90)) < 0.02).astype(np.uint8)

    def dev_sets():
        return [core.device_set(fa).alloc_outputs(want_stack=False),
                core.device_set(fb, mask=mask).alloc_outputs(want_stack=False),
                core.device_set(fc).alloc_outputs(want_stack=False)]

    def outs(sets):
        return [dict(mean=s.mean.cpu().numpy(), median=s.median.cpu().numpy(),
                     nkept=s.nkept.cpu().numpy().astype(np.int32)) for s in sets]

    alone = []
    for s in dev_sets():
        ws = core.reduce_sets([s], core.reduce_params("bilinear", core.clip_params(2.5, 3)))
        assert core.sync_status(ws) == 0
        alone += outs([s])
    for persistent in (False, True):
        sets = dev_sets()
        ws = core.reduce_sets(sets, core.reduce_params("bilinear", core.clip_params(2.5, 3),
                                                       persistent=persistent))
        assert core.sync_status(ws) == 0
        for a, b in zip(alone, outs(sets)):
            for key in ("mean", "median", "nkept"):
                assert np.array_equal(a[key].view(np.uint8), b[key].view(np.uint8)), key
    for fs, got in ((fa, alone[0]), (fc, alone[2])):
        ref = oracle.reduce_set(fs, interp="bilinear", kappa=2.5)
        samp = sample_tolerance(fs, "bilinear", oracle).max(axis=0)
        print(gate_e2e("window forms", got, ref, samp, 2.5))


def _padded_device_set(fs, pad_raw, pad_master):
    """Device set whose raw frames and masters are views into wider buffers
    (row pitch W + pad), so that neither need be 16-byte aligned per row."""
    n, H, W = fs.raw.shape
    big = torch.zeros((n, H, W + pad_raw), dtype=torch.uint16, device="cuda")
    big[..., :W] = torch.from_numpy(fs.raw.astype(np.int32)).to(torch.uint16).cuda()
    ms = []
    for a in (fs.bias, fs.dark, fs.flat):
        m = torch.ones((H, W + pad_master), dtype=torch.float32, device="cuda")
        m[:, :W] = torch.from_numpy(a).cuda()
        ms.append(m[:, :W])
    s = core.device_set(fs, raw=big[..., :W], masters=tuple(ms)).alloc_outputs(want_stack=True)
    s._keep.append(big)
    return s


@pytest.mark.parametrize("W,H,n,pad_raw,pad_master", [
    (1100, 37, 18, 0, 0),    # 64 columns per lane, two frame chunks, ragged row block
    (1021, 35, 5, 3, 1),     # unaligned raw and master rows
    (2048, 36, 3, 0, 0),     # widest row pass
    (96, 34, 17, 8, 4),      # narrow: most lanes past the frame
    (64, 300, 3, 0, 0),      # two column-pass row blocks, the second mostly mirrored
    (200, 513, 2, 4, 0),     # three row blocks with a one-row tail
    (1020, 40, 4, 0, 0),     # the paper's 1020 columns: 8-byte rows, partial last lane
    (1000, 36, 3, 0, 0),     # 16-byte rows, the last lane's chunks partly past the row
    (1018, 36, 3, 2, 0),     # 8-byte rows, a chunk cut inside its first half
])
@pytest.mark.parametrize("onchip", [False, True])
def test_spline_row_pass_shapes(W, H, n, pad_raw, pad_master, onchip):
    fs = synth.make_set(W, H, n, 6.0, 4100 + W + n, n_stars=30, n_cr=6)
    s = _padded_device_set(fs, pad_raw, pad_master)
    ws = core.reduce_sets([s], core.reduce_params("spline3", core.clip_params(3.0, 3),
                                                  spline_onchip=onchip))
    assert core.sync_status(ws) == 0
    got = dict(mean=s.mean.cpu().numpy(), median=s.median.cpu().numpy(),
               nkept=s.nkept.cpu().numpy().astype(np.int32), stack=s.stack.cpu().numpy())
    check_against_oracle(fs, got, "spline3", 3.0, 3)


def test_spline_batch_invariance_and_persistent():
    fss = [synth.make_set(80, 72, n, 6.0, 300 + n, n_stars=20, n_cr=4) for n in (4, 11)]
    alone = [run_fused([fs], "spline3", want_stack=False)[0] for fs in fss]
    batch = run_fused(fss, "spline3", persistent=True, want_stack=False)
    for a, b in zip(alone, batch):
        assert np.array_equal(a["mean"].view(np.uint32), b["mean"].view(np.uint32))
        assert np.array_equal(a["median"].view(np.uint32), b["median"].view(np.uint32))


def test_spline_batch_mixing_coefficient_paths():
    """One bucket holding sets on both spline paths (tiled prefilter for a
    30-row frame, row + column passes for the others): each equals its
    standalone reduction and the oracle."""
    fss = [synth.make_set(70, 30, 5, 5.0, 510, n_stars=12, n_cr=3),
           synth.make_set(70, 50, 5, 5.0, 511, n_stars=12, n_cr=3),
           synth.make_set(40, 36, 6, 5.0, 512, n_stars=12, n_cr=3)]
    alone = [run_fused([fs], "spline3", want_stack=False)[0] for fs in fss]
    batch = run_fused(fss, "spline3", want_stack=False)
    for fs, a, b in zip(fss, alone, batch):
        assert np.array_equal(a["mean"].view(np.uint32), b["mean"].view(np.uint32))
        assert np.array_equal(a["median"].view(np.uint32), b["median"].view(np.uint32))
        ref = oracle.reduce_set(fs, interp="spline3")
        samp = sample_tolerance(fs, "spline3", oracle).max(axis=0)
        gate_e2e("mixed spline", b, ref, samp, 3.0)


def test_normalize_flat():
    fs = synth.make_set(70, 50, 6, 3.0, 41, n_stars=20)
    fs.flat = (fs.flat * 1.7).astype(np.float32)   # not normalised to 1
    got = run_fused([fs], "bilinear", normalize_flat=True)[0]
    check_against_oracle(fs, got, "bilinear", 3.0, 3, normalize_flat=True)


def test_clip_options_median_centre_and_ddof():
    fs = synth.make_set(64, 48, 21, 3.0, 77, n_stars=20, n_cr=30)
    for center, ddof in (("median", 0), ("mean", 1)):
        got = run_fused([fs], "bilinear", kappa=2.0, center=center, ddof=ddof)[0]
        st = got["stack"]
        gvalid = ~np.isnan(st)
        same = oracle.combine_stack(np.where(gvalid, st, 0.0), gvalid, kappa=2.0, center=center,
                                    ddof=ddof)
        ok = (got["nkept"] == same["nkept"]) | (same["margin"] < 1e-5)
        assert ok.all()
        compare("clip option mean", got["mean"], same["mean"], mean_tolerance(same["mean"]),
                got["nkept"] == same["nkept"])


# ------------------------------------------------------------- edge cases
@pytest.mark.parametrize("interp", ["nearest", "bilinear", "spline3", "cubic"])
def test_edge_shapes_and_offsets(interp):
    cases = [
        synth.make_const_set(1, 1, 1, 1500, 1000.0, 0.05, 0.8, 60.0),
        synth.make_const_set(9, 5, 2, 1500, 1000.0, 0.05, 0.8, 60.0, dx=[0.5, -0.5], dy=[0.0, 0.5]),
        synth.make_set(9, 33, 3, 1.0, 5, n_stars=3, n_cr=1),
        synth.make_set(40, 17, 2, 0.0, 6, n_stars=3, n_cr=1),
    ]
    # integer offsets: pure pixel moves; huge offsets: no valid sample at all
    fs = synth.make_set(37, 19, 4, 0.0, 8, n_stars=5, n_cr=2)
    fs.dx = np.array([0.0, 3.0, -2.0, 1.0])
    fs.dy = np.array([0.0, -1.0, 2.0, 4.0])
    cases.append(fs)
    far = synth.make_set(20, 20, 3, 0.0, 9, n_stars=2, n_cr=0)
    far.dx = np.array([50.0, -60.5, 1e6])
    far.dy = np.array([0.0, 0.0, 0.0])
    cases.append(far)
    for fs in cases:
        got = run_fused([fs], interp)[0]
        ref = oracle.reduce_set(fs, interp=interp, want_stack=True)
        assert np.array_equal(~np.isnan(got["stack"]), ref["valid"])
        assert np.array_equal(got["nkept"], ref["nkept"])
        assert np.array_equal(np.isnan(got["mean"]), np.isnan(ref["mean"]))
        tol = sample_tolerance(fs, interp, oracle).max(axis=0) + mean_tolerance(ref["mean"])
        compare("edge mean", got["mean"], ref["mean"], tol)
    # integer shifts with bilinear/nearest are exact pixel moves of the calibrated frame
    if interp != "spline3":
        fs = cases[4]
        got = run_fused([fs], interp)[0]
        v1 = got["stack"][1]
        v0 = got["stack"][0]
        # frame 1 sampled at (x+3, y-1) equals frame 1's own calibration: compare with
        # the identity-offset stack entry of a second run
        fs2 = synth.FrameSet(raw=fs.raw[1:2], bias=fs.bias, dark=fs.dark, flat=fs.flat,
                             exptime=fs.exptime[1:2], dx=np.zeros(1), dy=np.zeros(1))
        ident = run_fused([fs2], interp)[0]["stack"][0]
        H, W = v1.shape
        assert np.array_equal(v1[1:, :W - 3], ident[:H - 1, 3:])
        assert np.isnan(v0).sum() == 0


def test_all_invalid_pixels_are_nan():
    far = synth.make_set(20, 20, 3, 0.0, 9, n_stars=2, n_cr=0)
    far.dx = np.array([500.0, -600.5, 1e6])
    got = run_fused([far], "bilinear")[0]
    assert np.isnan(got["mean"]).all() and np.isnan(got["median"]).all()
    assert (got["nkept"] == 0).all()


# ------------------------------------------------------------ status paths
def test_bad_flat_master_is_latched():
    fs = synth.make_set(40, 30, 3, 1.0, 10, n_stars=3)
    fs.flat[5, 7] = 0.0
    s = core.device_set(fs).alloc_outputs()
    ws = core.reduce_sets([s], core.reduce_params("bilinear"))
    assert core.sync_status(ws) == 5
    assert core.sync_status(ws) == 0  # cleared after reading


@pytest.mark.parametrize("interp,H", [("bilinear", 32), ("spline3", 32), ("spline3", 40)])
def test_bounded_wait_gives_up_with_timeout(interp, H):
    """A set whose ready flag nothing sets: the kernels' bounded waits end
    (the spline prefilter's too: 32 rows take the tiled prefilter, 40 the
    row pass), IRP_ERR_TIMEOUT is latched, and the context stays usable."""
    fs = synth.make_set(64, H, 3, 1.0, 11, n_stars=3)
    s = core.device_set(fs).alloc_outputs()
    s.ready_flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    s.ready_value = 1
    ws = core.reduce_sets([s], core.reduce_params(interp, wait_spin_limit=2000))
    assert core.sync_status(ws) == 7
    s.ready_flag.fill_(1)
    ws = core.reduce_sets([s], core.reduce_params(interp, wait_spin_limit=2000), ws=ws)
    assert core.sync_status(ws) == 0
    ref = oracle.reduce_set(fs, interp=interp)
    got = dict(mean=s.mean.cpu().numpy(), median=s.median.cpu().numpy(),
               nkept=s.nkept.cpu().numpy())
    gate_e2e("after timeout", got, ref, sample_tolerance(fs, interp, oracle).max(axis=0), 3.0)


def test_plan_launch_and_graph_capture():
    fss = [synth.make_set(96, 64, n, 4.0, 60 + n, n_stars=10) for n in (5, 12, 30)]
    sets = [core.device_set(fs).alloc_outputs() for fs in fss]
    params = core.reduce_params("bilinear", persistent=True)
    plan = core.Plan(sets, params)
    plan.launch()
    torch.cuda.synchronize()
    first = [s.mean.clone() for s in sets]
    for s in sets:
        s.mean.zero_()
    g = torch.cuda.CUDAGraph()
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            plan.launch(stream=stream)
    g.replay()
    torch.cuda.synchronize()
    for a, s in zip(first, sets):
        assert torch.equal(a.view(torch.int32), s.mean.view(torch.int32))
    assert core.sync_status(plan.ws) == 0


# --------------------------------------------------------------- unfused path
@pytest.mark.parametrize("W", [90, 96])  # scalar rows / 8-pixel vector rows
@pytest.mark.parametrize("interp", ["nearest", "bilinear", "spline3", "cubic"])
def test_unfused_f32_matches_oracle(interp, W):
    fs = synth.make_set(W, 66, 9, 4.0, 123, n_stars=30, n_cr=10)
    d = core.device_set(fs)
    raw = torch.stack(d.frames)
    cal, _, _, _ = core.calibrate(raw, d.bias, d.dark, d.flat, fs.exptime)
    cal_h = cal.cpu().numpy()
    for k in range(fs.n):
        v = oracle.calibrate(fs.raw[k], fs.bias, fs.dark, fs.flat, fs.exptime[k])
        lv = np.abs(fs.bias.astype(np.float64) + fs.dark.astype(np.float64) * fs.exptime[k])
        compare("calibrate", cal_h[k], v,
                4 * 2.0 ** -24 * (np.abs(v) + lv / fs.flat.astype(np.float64)) + 1e-5)
    stack, valid, _ = core.shift(cal, fs.dx, fs.dy, interp)
    st = stack.cpu().numpy()
    va = valid.cpu().numpy().astype(bool)
    assert np.array_equal(va, ~np.isnan(st))
    for k in range(fs.n):
        a, ok = oracle.shift(cal_h[k].astype(np.float64), fs.dx[k], fs.dy[k], interp)
        assert np.array_equal(ok, va[k])
        M = np.abs(cal_h[k]).max()
        coef = {"spline3": 64, "cubic": 16}.get(interp, 8)
        compare("shift", np.where(ok, st[k], np.nan), np.where(ok, a, np.nan),
                coef * 2.0 ** -24 * M + 1e-4)
    out = core.combine(stack, valid=valid, clip=core.clip_params(2.5), want_reject=True)
    same = oracle.combine_stack(np.where(va, st, 0.0), va, kappa=2.5)
    med = out["median"].cpu().numpy()
    fin = ~np.isnan(same["median"])
    assert np.array_equal(med[fin].view(np.uint32), same["median"].astype(np.float32)[fin].view(np.uint32))
    kept = out["nkept"].cpu().numpy().astype(np.int32)
    exempt = same["margin"] < 1e-5
    assert ((kept == same["nkept"]) | exempt).all()
    rej = out["reject"].cpu().numpy().astype(bool)
    assert ((rej == same["rejected"]).all(axis=0) | exempt).all()
    compare("combine mean", out["mean"].cpu().numpy(), same["mean"], mean_tolerance(same["mean"]),
            kept == same["nkept"])


@pytest.mark.parametrize("interp", ["bilinear", "spline3"])
def test_unfused_f16_scaled_stack(interp):
    """FP16 stack with per-frame power-of-two scale and FP64-mean offset."""
    fs = synth.make_set(80, 60, 8, 4.0, 124, n_stars=30, n_cr=10)
    d = core.device_set(fs)
    raw = torch.stack(d.frames)
    h, scale, offset, _ = core.calibrate(raw, d.bias, d.dark, d.flat, fs.exptime, dtype="f16")
    sc = scale.cpu().numpy()
    of = offset.cpu().numpy()
    hh = h.cpu().numpy().astype(np.float32)
    for k in range(fs.n):
        v = oracle.calibrate(fs.raw[k], fs.bias, fs.dark, fs.flat, fs.exptime[k])
        assert of[k] == pytest.approx(v.mean(), rel=1e-6, abs=1e-3)
        assert np.abs((v - of[k]) / sc[k]).max() <= 16384.0
        assert sc[k] == 2.0 ** np.round(np.log2(sc[k]))
        deq = hh[k] * sc[k] + of[k]
        # half has 11 significant bits: relative rounding 2^-11 of |v - offset|
        compare("f16 calibrate", deq, v, 2.0 ** -11 * np.abs(v - of[k]) + 1e-3 + 1e-6 * np.abs(v))
    stack, valid, _ = core.shift(h, fs.dx, fs.dy, interp, dtype="f16", scale=scale, offset=offset)
    out = core.combine(stack, dtype="f16", scale=scale, offset=offset, valid=valid,
                       clip=core.clip_params(3.0))
    st = stack.cpu().numpy().astype(np.float32)
    va = valid.cpu().numpy().astype(bool)
    deq = st * sc[:, None, None] + of[:, None, None]
    same = oracle.combine_stack(np.where(va, deq, 0.0), va, kappa=3.0)
    med = out["median"].cpu().numpy()
    fin = ~np.isnan(same["median"])
    assert np.array_equal(med[fin].view(np.uint32), same["median"].astype(np.float32)[fin].view(np.uint32))
    ref = oracle.reduce_set(fs, interp=interp)
    m = (ref["margin"] >= 1e-2) & (out["nkept"].cpu().numpy() == ref["nkept"])
    err = np.abs(out["mean"].cpu().numpy() - ref["mean"])[m]
    # reported, bounded by the FP16 quantisation of |v - offset| (2^-11 relative)
    assert np.all(err <= 2.0 ** -10 * np.abs(ref["mean"][m] - of.mean()) + 0.05 + 1e-3 * np.abs(ref["mean"][m]))


def test_frame_stats_f64():
    fs = synth.make_set(300, 200, 4, 2.0, 125, n_stars=30)
    d = core.device_set(fs)
    cal, _, _, _ = core.calibrate(torch.stack(d.frames), d.bias, d.dark, d.flat, fs.exptime)
    s, q, c = core.frame_stats(cal)
    h = cal.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(s.cpu().numpy(), h.reshape(4, -1).sum(1), rtol=1e-12)
    np.testing.assert_allclose(q.cpu().numpy(), (h ** 2).reshape(4, -1).sum(1), rtol=1e-12)
    assert (c.cpu().numpy() == 300 * 200).all()


def test_frame_stats_f64_wide_rows():
    """Rows of 4100 pixels (17 values per thread and row) with bright stars and
    cosmic rays: the per-row FP32 partials with exact error terms keep the
    FP64 accuracy of the frame sums."""
    fs = synth.make_set(4100, 24, 3, 2.0, 126, n_stars=400, n_cr=200)
    d = core.device_set(fs)
    cal, _, _, _ = core.calibrate(torch.stack(d.frames), d.bias, d.dark, d.flat, fs.exptime)
    s, q, c = core.frame_stats(cal)
    h = cal.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(s.cpu().numpy(), h.reshape(3, -1).sum(1), rtol=1e-12)
    np.testing.assert_allclose(q.cpu().numpy(), (h ** 2).reshape(3, -1).sum(1), rtol=1e-12)
    assert (c.cpu().numpy() == 4100 * 24).all()


# ------------------------------------------------ bad-pixel masking (Sec. 2.1)
@pytest.mark.parametrize("interp", ["nearest", "bilinear", "spline3", "cubic"])
@pytest.mark.parametrize("offset", [4.0, 40.0])   # union master window / masters from HBM
def test_masked_reduction_matches_oracle(interp, offset):
    fs = synth.make_set(101, 77, 14, offset, 1313, n_stars=40, n_cr=10)
    rng = np.random.default_rng(5)
    mask = (rng.random((77, 101)) < 0.02).astype(np.uint8)
    sat = 20000.0
    s = core.device_set(fs, mask=mask, saturation=sat).alloc_outputs(want_stack=True)
    ws = core.reduce_sets([s], core.reduce_params(interp, core.clip_params(2.5, 3)))
    assert core.sync_status(ws) == 0
    ref = oracle.reduce_set(fs, interp=interp, kappa=2.5, mask=mask, saturation=sat,
                            want_stack=True)
    st = s.stack.cpu().numpy()
    gvalid = ~np.isnan(st)
    assert np.array_equal(gvalid, ref["valid"]), "masked validity differs"
    assert (~ref["valid"]).sum() > (~oracle.reduce_set(fs, interp=interp, want_stack=True)["valid"]).sum()
    tol = sample_tolerance(fs, interp, oracle)
    compare("masked stack", st, np.where(ref["valid"], ref["stack"], np.nan), tol)
    got = dict(mean=s.mean.cpu().numpy(), median=s.median.cpu().numpy(),
               nkept=s.nkept.cpu().numpy())
    samp = np.max(np.where(ref["valid"], tol, 0.0), axis=0)
    meas = np.max(np.where(ref["valid"], np.abs(np.where(gvalid, st, 0.0) - ref["stack"]), 0.0),
                  axis=0)
    print(gate_e2e("masked", got, ref, samp, 2.5, meas=meas))


# ------------------------------------------- overscan cutout (Sec. 2.1 geometry)
@pytest.mark.parametrize("interp", ["bilinear", "spline3"])
def test_overscan_cutout_roi_of_1074x1024_frames(interp):
    """Raw frames of 1074x1024 with a 50-column overscan and 2 px trimmed on
    every side leave 1020x1020 (Sec. 2.1): the cutout is a region of the raw
    and master buffers (pointer offset, pitch 1074), reduced in place; it must
    equal the reduction of the same region copied out."""
    full = synth.make_set(1074, 1024, 4, 5.0, 10741024, n_stars=120, n_cr=10)
    x0, y0, W, H = 52, 2, 1020, 1020
    fs = synth.FrameSet(raw=np.ascontiguousarray(full.raw[:, y0:y0 + H, x0:x0 + W]),
                        bias=np.ascontiguousarray(full.bias[y0:y0 + H, x0:x0 + W]),
                        dark=np.ascontiguousarray(full.dark[y0:y0 + H, x0:x0 + W]),
                        flat=np.ascontiguousarray(full.flat[y0:y0 + H, x0:x0 + W]),
                        exptime=full.exptime, dx=full.dx, dy=full.dy)
    raw_dev = torch.from_numpy(full.raw.astype(np.int32)).to(torch.uint16).cuda()
    masters = [torch.from_numpy(a).cuda()[y0:y0 + H, x0:x0 + W]
               for a in (full.bias, full.dark, full.flat)]
    s = core.device_set(fs, raw=raw_dev[:, y0:y0 + H, x0:x0 + W], masters=tuple(masters))
    assert s.frames[0].stride(0) == 1074 and s.bias.stride(0) == 1074
    s.alloc_outputs(want_stack=False)
    ws = core.reduce_sets([s], core.reduce_params(interp))
    assert core.sync_status(ws) == 0
    copied = run_fused([fs], interp, want_stack=False)[0]
    assert np.array_equal(s.mean.cpu().numpy().view(np.uint32), copied["mean"].view(np.uint32))
    assert np.array_equal(s.median.cpu().numpy().view(np.uint32), copied["median"].view(np.uint32))
    rng = np.random.default_rng(7)
    xs, ys = rng.integers(0, W, 3000), rng.integers(0, H, 3000)
    ref = oracle.reduce_set(fs, interp=interp, pixels=(xs, ys), nthreads=os.cpu_count() or 1)
    samp = sample_tolerance(fs, interp, oracle).max(axis=0)[ys, xs]
    g = dict(mean=s.mean.cpu().numpy()[ys, xs], median=s.median.cpu().numpy()[ys, xs],
             nkept=s.nkept.cpu().numpy()[ys, xs])
    print(gate_e2e("cutout", g, ref, samp, 3.0))


@pytest.mark.parametrize("W,onchip", [(2049, False), (4100, False), (4100, True), (6000, False)])
def test_spline_rows_wider_than_2048_in_segments(W, onchip):
    """Rows wider than 2048 columns take the row pass in overlapping segments
    (64-column halos, recursions started at the segment's ends); every
    sample, and the combined outputs, match the oracle's whole-row solve."""
    fs = synth.make_set(W, 40, 3, 8.0, 7700 + W, n_stars=40, n_cr=6)
    got = run_fused([fs], "spline3", kappa=2.5, onchip=onchip)[0]
    print(W, onchip, check_against_oracle(fs, got, "spline3", 2.5, 3))


def test_masked_spline_rows_wider_than_2048():
    fs = synth.make_set(4100, 40, 4, 8.0, 7790, n_stars=40, n_cr=6)
    rng = np.random.default_rng(77)
    mask = (rng.random((40, 4100)) < 0.01).astype(np.uint8)
    s = core.device_set(fs, mask=mask, saturation=20000.0).alloc_outputs(want_stack=True)
    ws = core.reduce_sets([s], core.reduce_params("spline3", core.clip_params(2.5, 3)))
    assert core.sync_status(ws) == 0
    ref = oracle.reduce_set(fs, interp="spline3", kappa=2.5, mask=mask, saturation=20000.0,
                            want_stack=True)
    st = s.stack.cpu().numpy()
    assert np.array_equal(~np.isnan(st), ref["valid"]), "masked validity differs"
    tol = sample_tolerance(fs, "spline3", oracle)
    compare("wide masked stack", st, np.where(ref["valid"], ref["stack"], np.nan), tol)


def test_spline_tile_stripes_of_a_set_larger_than_the_l2_budget():
    """A set whose row-pass coefficients exceed the share of L2 the launch
    sequence keeps them in (12 frames of 2048 x 640: 63 MB) is reduced in
    stripes of rows; the pixels on both sides of every stripe boundary, and a
    random sample, match the oracle."""
    W, H, n = 2048, 640, 12
    fs = synth.make_set(W, H, n, 10.0, 2048640, n_stars=300, n_cr=20)
    got = run_fused([fs], "spline3", want_stack=False, onchip=True)[0]
    rng = np.random.default_rng(64)
    band = np.arange(200, 320)  # around the first stripe ends (256 rows, less warm-up)
    band2 = np.arange(440, 580)
    rows = np.concatenate([band, band2, [0, 1, H - 2, H - 1]])
    xs = np.concatenate([np.tile(np.arange(0, W, 16), rows.size), rng.integers(0, W, 4000)])
    ys = np.concatenate([np.repeat(rows, W // 16), rng.integers(0, H, 4000)])
    ref = oracle.reduce_set(fs, interp="spline3", pixels=(xs, ys), nthreads=os.cpu_count() or 1)
    g = {k: got[k][ys, xs] for k in ("mean", "median", "nkept")}
    samp = sample_tolerance(fs, "spline3", oracle, pixels=(xs, ys)).max(axis=0)
    print(gate_e2e("spline stripes", g, ref, samp, 3.0))


def test_masked_spline_edges_and_integer_shifts():
    """Masked cubic spline at the frame edges (the footprint mirrored there)
    and with integer offsets, where the fourth tap of an axis has zero weight
    and the footprint is 3 taps wide: validity bit-exact against the oracle."""
    fs = synth.make_set(70, 45, 6, 3.0, 4545, n_stars=15, n_cr=5)
    fs.dx = np.array([0.0, 2.0, -1.0, 0.5, -2.25, 1.75])
    fs.dy = np.array([0.0, -1.0, 3.0, 0.0, 1.5, -0.5])
    mask = np.zeros((45, 70), np.uint8)
    mask[0, 5] = mask[1, 30] = mask[44, 10] = mask[20, 0] = mask[22, 69] = mask[10, 40] = 1
    mask[30:32, 50:52] = 1
    s = core.device_set(fs, mask=mask, saturation=30000.0).alloc_outputs(want_stack=True)
    ws = core.reduce_sets([s], core.reduce_params("spline3", core.clip_params(3.0, 3)))
    assert core.sync_status(ws) == 0
    ref = oracle.reduce_set(fs, interp="spline3", mask=mask, saturation=30000.0, want_stack=True)
    st = s.stack.cpu().numpy()
    assert np.array_equal(~np.isnan(st), ref["valid"]), "masked spline validity differs"
    tol = sample_tolerance(fs, "spline3", oracle)
    compare("masked spline stack", st, np.where(ref["valid"], ref["stack"], np.nan), tol)

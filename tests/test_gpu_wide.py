"""GPU parity of sets deeper than the register buckets (65 to 1024 frames; the
paper's bands hold 180 frames each, Sec. 2.1): the warp-per-pixel combine
through irp_combine, and irp_reduce_set, which resamples such a set into its
aligned stack chunk by chunk and then combines it.  Everything is compared
with the oracle element by element."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2008_11486_gb300 import build as irp_build
from paper_2008_11486_gb300 import core, synth
from parity_util import compare, gate_e2e, mean_tolerance, sample_tolerance
from test_gpu_parity import check_against_oracle, run_fused

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _native():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    irp_build.build()


def deep_stack(n, H, W, seed, invalid_frac=0.05):
    """Aligned FP32 stack [n, H, W]: sky-like Gaussian samples, cosmic-ray
    outliers, bright pixels near saturation, NaN (invalid) samples, a pixel
    with no valid sample, one with a single sample and one of equal values."""
    rng = np.random.default_rng(seed)
    st = (300.0 + 10.0 * rng.standard_normal((n, H, W))).astype(np.float32)
    cr = rng.random((n, H, W)) < 0.02
    st[cr] += rng.uniform(5e3, 3e4, int(cr.sum())).astype(np.float32)
    st[:, 0, :5] += np.float32(6.0e4)
    st[rng.random((n, H, W)) < invalid_frac] = np.nan
    st[:, 1, 0] = np.nan
    st[1:, 1, 1] = np.nan
    st[0, 1, 1] = 42.0
    st[:, 2, 2] = 123.5
    return st


def check_combine(st, out, **clip):
    va = ~np.isnan(st)
    same = oracle.combine_stack(np.where(va, st, 0.0), va, **clip)
    med = out["median"].cpu().numpy()
    assert np.array_equal(np.isnan(med), np.isnan(same["median"]))
    fin = ~np.isnan(same["median"])
    assert np.array_equal(med[fin].view(np.uint32),
                          same["median"].astype(np.float32)[fin].view(np.uint32))
    kept = out["nkept"].cpu().numpy().astype(np.int32)
    exempt = same["margin"] < 1e-5
    assert exempt.mean() < 1e-2
    assert ((kept == same["nkept"]) | exempt).all()
    if out.get("reject") is not None:
        rej = out["reject"].cpu().numpy().astype(bool)
        assert ((rej == same["rejected"]).all(axis=0) | exempt).all()
    mean = out["mean"].cpu().numpy()
    assert np.array_equal(np.isnan(mean), np.isnan(same["mean"]))
    return compare("wide mean", mean, same["mean"], mean_tolerance(same["mean"]),
                   (kept == same["nkept"]) & fin)


@pytest.mark.parametrize("n", [65, 100, 128, 129, 180, 256, 257, 511, 513, 1024])
def test_wide_combine_frame_counts(n):
    st = deep_stack(n, 5, 45, 7000 + n)  # two 32-pixel tiles per row, the second ragged
    out = core.combine(torch.from_numpy(st).cuda(), clip=core.clip_params(3.0, 3),
                       want_reject=True)
    print(n, check_combine(st, out, kappa=3.0, max_iter=3))


@pytest.mark.parametrize("clip", [
    dict(kappa=2.5, max_iter=10),
    dict(kappa=3.0, max_iter=3, center="median"),
    dict(kappa=3.0, max_iter=5, ddof=1),
    dict(kappa=3.0, max_iter=4, kappa_lo=2.0, kappa_hi=4.0),
    dict(kappa=3.0, max_iter=0),
])
def test_wide_combine_clip_options(clip):
    st = deep_stack(150, 6, 33, 7100)
    out = core.combine(torch.from_numpy(st).cuda(), clip=core.clip_params(**clip),
                       want_reject=True)
    check_combine(st, out, **clip)


def test_wide_combine_valid_mask_and_f16():
    n, H, W = 200, 4, 40
    st = deep_stack(n, H, W, 7200, invalid_frac=0.0)
    rng = np.random.default_rng(7201)
    valid = rng.random((n, H, W)) >= 0.1
    out = core.combine(torch.from_numpy(st).cuda(),
                       valid=torch.from_numpy(valid.astype(np.uint8)).cuda())
    check_combine(np.where(valid, st, np.nan).astype(np.float32), out, kappa=3.0, max_iter=3)
    # FP16 stack with per-frame scale and offset: the combine sees h * scale + offset
    # per-frame offset, and the smallest power-of-two scale keeping |h| <= 16384
    offset = rng.uniform(250, 350, n).astype(np.float32)
    span = np.nanmax(np.abs(st - offset[:, None, None]), axis=(1, 2))
    scale = (2.0 ** np.ceil(np.log2(span / 16384.0))).astype(np.float32)
    h = ((np.nan_to_num(st, nan=0.0) - offset[:, None, None]) /
         scale[:, None, None]).astype(np.float16)
    deq = h.astype(np.float32) * scale[:, None, None] + offset[:, None, None]
    deq = np.where(np.isnan(st), np.nan, deq).astype(np.float32)
    hh = torch.from_numpy(np.where(np.isnan(st), np.float16(np.nan), h)).cuda()
    out = core.combine(hh, dtype="f16", scale=torch.from_numpy(scale).cuda(),
                       offset=torch.from_numpy(offset).cuda())
    check_combine(deq, out, kappa=3.0, max_iter=3)


# ------------------------------------------------------- fused irp_reduce_set
@pytest.mark.parametrize("interp,W,H,n", [
    ("bilinear", 70, 40, 100),
    ("nearest", 45, 30, 65),
    ("spline3", 40, 36, 80),    # row + column coefficient passes
    ("spline3", 30, 20, 70),    # tiled coefficient path (W, H < 34)
    ("bilinear", 50, 20, 300),
])
def test_deep_set_fused_matches_oracle(interp, W, H, n):
    fs = synth.make_set(W, H, n, 5.0, 7300 + n, n_stars=15, n_cr=4)
    got = run_fused([fs], interp, kappa=3.0)[0]
    check_against_oracle(fs, got, interp, 3.0, 3)


@pytest.mark.parametrize("W,H,n", [(40, 36, 80), (100, 50, 200), (70, 34, 65)])
def test_deep_spline_from_filtered_rows_equals_stack_path(W, H, n):
    """Without a caller stack, a deep spline set is combined straight from its
    horizontally filtered rows (vertical taps inside the combine); with one,
    its chunks write the stack first.  The samples are formed by the same
    FP32 operations, so the two results are bit-identical."""
    fs = synth.make_set(W, H, n, 5.0, 7350 + n, n_stars=15, n_cr=4)
    rows = run_fused([fs], "spline3", want_stack=False)[0]
    stack = run_fused([fs], "spline3", want_stack=True)[0]
    for k in ("mean", "median"):
        assert np.array_equal(rows[k].view(np.uint32), stack[k].view(np.uint32)), k
    assert np.array_equal(rows["nkept"], stack["nkept"])
    ref = oracle.reduce_set(fs, interp="spline3")
    samp = sample_tolerance(fs, "spline3", oracle).max(axis=0)
    print(gate_e2e("deep spline rows", rows, ref, samp, 3.0))


def test_deep_set_in_a_batch_and_persistent():
    """A deep set (workspace stack) beside plain sets: each result equals its
    standalone reduction, in both launch forms."""
    fss = [synth.make_set(64, 40, 90, 4.0, 7400, n_stars=10, n_cr=3),
           synth.make_set(50, 30, 12, 4.0, 7401, n_stars=10, n_cr=3),
           synth.make_set(33, 70, 66, 4.0, 7402, n_stars=10, n_cr=3)]
    alone = [run_fused([fs], "bilinear", want_stack=False)[0] for fs in fss]
    for persistent in (False, True):
        batch = run_fused(fss, "bilinear", persistent=persistent, want_stack=False)
        for a, b in zip(alone, batch):
            for k in ("mean", "median"):
                assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32))
            assert np.array_equal(a["nkept"], b["nkept"])
    # the workspace-stack form equals the caller-stack form
    with_stack = run_fused(fss[:1], "bilinear", want_stack=True)[0]
    assert np.array_equal(with_stack["mean"].view(np.uint32), alone[0]["mean"].view(np.uint32))


def test_deep_spline_sets_in_a_batch():
    """Two deep spline sets (filtered-row path, and the tiled path's stack
    chunks for a 30-row frame) beside a plain one, in both launch forms."""
    fss = [synth.make_set(64, 40, 90, 4.0, 7410, n_stars=10, n_cr=3),
           synth.make_set(50, 30, 70, 4.0, 7411, n_stars=10, n_cr=3),
           synth.make_set(48, 48, 9, 4.0, 7412, n_stars=10, n_cr=3)]
    alone = [run_fused([fs], "spline3", want_stack=False)[0] for fs in fss]
    for persistent in (False, True):
        batch = run_fused(fss, "spline3", persistent=persistent, want_stack=False)
        for a, b in zip(alone, batch):
            for k in ("mean", "median"):
                assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32))


def test_deep_set_masked():
    fs = synth.make_set(60, 30, 96, 4.0, 7500, n_stars=20, n_cr=5)
    rng = np.random.default_rng(7501)
    mask = (rng.random((30, 60)) < 0.02).astype(np.uint8)
    s = core.device_set(fs, mask=mask, saturation=20000.0).alloc_outputs(want_stack=True)
    ws = core.reduce_sets([s], core.reduce_params("bilinear", core.clip_params(3.0, 3)))
    assert core.sync_status(ws) == 0
    ref = oracle.reduce_set(fs, interp="bilinear", mask=mask, saturation=20000.0, want_stack=True)
    st = s.stack.cpu().numpy()
    assert np.array_equal(~np.isnan(st), ref["valid"])
    got = dict(mean=s.mean.cpu().numpy(), median=s.median.cpu().numpy(),
               nkept=s.nkept.cpu().numpy())
    samp = sample_tolerance(fs, "bilinear", oracle).max(axis=0)
    meas = np.max(np.where(ref["valid"], np.abs(np.nan_to_num(st) - ref["stack"]), 0.0), axis=0)
    print(gate_e2e("deep masked", got, ref, samp, 3.0, meas=meas))


def test_paper_band_180_frames_sampled():
    """One band of the paper's run: 180 frames of 1020x1020, spline shift
    (Sec. 2.1); random pixels and every 7th pixel of two edges against the
    oracle."""
    fs = synth.make_set(1020, 1020, 180, 10.0, 7600, n_stars=200, n_cr=20)
    got = run_fused([fs], "spline3", want_stack=False)[0]
    rng = np.random.default_rng(7601)
    W = H = 1020
    xs = np.concatenate([rng.integers(0, W, 1500), np.arange(0, W, 7), np.zeros(H // 7 + 1, int)])
    ys = np.concatenate([rng.integers(0, H, 1500), np.zeros(W // 7 + 1, int), np.arange(0, H, 7)])
    ref = oracle.reduce_set(fs, interp="spline3", pixels=(xs, ys), nthreads=os.cpu_count() or 1)
    g = {k: got[k][ys, xs] for k in ("mean", "median", "nkept")}
    samp = sample_tolerance(fs, "spline3", oracle, pixels=(xs, ys)).max(axis=0)
    print(gate_e2e("paper band", g, ref, samp, 3.0))

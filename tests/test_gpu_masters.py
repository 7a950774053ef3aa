"""Master frames built on the GPU with the library's own calls (Sec. 2.1: the
frames are calibrated with bias, dark and flat masters).

Bias, dark and flat exposures are synthesised; each master is the
sigma-clipped mean (and median) of its calibrated exposures, formed with
irp_calibrate (bias subtracted; a dark exposure divided by its exposure time
through a constant flat equal to it) and irp_combine.  Each master is
compared with the oracle's calibration and combination of the same
exposures, and a science set is then reduced with the GPU's masters
(flat normalised by its FP64 mean) and compared with the oracle given the
same masters."""
import numpy as np
import pytest
import torch

import oracle
from paper_2008_11486_gb300 import build as irp_build
from paper_2008_11486_gb300 import core, synth
from parity_util import gate_e2e, mean_tolerance, sample_tolerance

pytestmark = pytest.mark.gpu

W, H = 160, 120


@pytest.fixture(scope="module", autouse=True)
def _native():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    irp_build.build()


def _exposures(rng, n, level, noise, t, n_cr=0):
    """n raw exposures: level [H, W] (ADU) + Gaussian read noise + cosmic rays."""
    raw = level[None] + rng.normal(0.0, noise, (n, H, W))
    for k in range(n):
        ys, xs = rng.integers(0, H, n_cr), rng.integers(0, W, n_cr)
        raw[k, ys, xs] += rng.uniform(5e3, 3e4, n_cr)
    return np.clip(np.round(raw), 0, 65535).astype(np.uint16)


def _gpu_master(raw, bias, dark, flat, t, kappa=3.0):
    """irp_calibrate of each exposure, then irp_combine of the stack."""
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    frames = torch.from_numpy(raw.astype(np.int32)).to(torch.uint16).cuda()
    cal, _, _, _ = core.calibrate(frames, d(bias), d(dark), d(flat), np.full(raw.shape[0], t))
    out = core.combine(cal, clip=core.clip_params(kappa, 3))
    torch.cuda.synchronize()
    return cal.cpu().numpy(), {k: out[k].cpu().numpy() for k in ("mean", "median", "nkept")}


def _oracle_master(raw, bias, dark, flat, t, kappa=3.0):
    st = np.stack([oracle.calibrate(r, bias, dark, flat, t) for r in raw])
    return st, oracle.combine_stack(st, np.ones(st.shape, np.uint8), kappa=kappa)


def _check(name, gcal, g, ocal, o, level=0.0):
    # identical calibrated inputs give the same median bit for bit
    same = oracle.combine_stack(gcal.astype(np.float64), np.ones(gcal.shape, np.uint8))
    assert np.array_equal(g["median"].view(np.uint32),
                          same["median"].astype(np.float32).view(np.uint32)), name
    # end to end against the oracle's FP64 calibration: a few roundings per
    # sample, of the calibrated value and of the level removed (bias + dark*t,
    # divided by the flat: `level`)
    samp = 8 * 2.0 ** -24 * (np.abs(ocal).max(axis=0) + level) + 1e-6
    return gate_e2e(name, g, o, samp, 3.0)


def test_bias_dark_flat_masters_with_irp_combine():
    rng = np.random.default_rng(21081)
    fs = synth.make_set(W, H, 6, 4.0, 2108, n_stars=30, n_cr=6)  # true masters and a science set
    zeros, ones = np.zeros((H, W), np.float32), np.ones((H, W), np.float32)
    # bias: 9 exposures of the bias level with read noise 10 ADU
    braw = _exposures(rng, 9, fs.bias.astype(np.float64), 10.0, 0.0, n_cr=3)
    gcal, gb = _gpu_master(braw, zeros, zeros, ones, 0.0)
    ocal, ob = _oracle_master(braw, zeros, zeros, ones, 0.0)
    print(_check("bias master", gcal, gb, ocal, ob))
    # with 9 exposures a 3-sigma clip cannot reject a lone cosmic ray (with
    # ddof 0 no sample lies beyond sqrt(n - 1) sigma): the median is the master
    bias_m = gb["median"]
    # dark: 7 exposures of 300 s; (raw - bias) / 300 through a constant flat of 300
    td = 300.0
    draw = _exposures(rng, 7, fs.bias + fs.dark.astype(np.float64) * td, 10.0, td, n_cr=8)
    tflat = np.full((H, W), td, np.float32)
    gcal, gd = _gpu_master(draw, bias_m, zeros, tflat, td)
    ocal, od = _oracle_master(draw, bias_m, zeros, tflat, td)
    print(_check("dark master", gcal, gd, ocal, od, np.abs(bias_m) / td))
    dark_m = gd["median"]  # 7 exposures: the median, as for the bias
    # flat: 11 twilight exposures of 5 s at 20000 e-
    tf = 5.0
    level = fs.bias + fs.dark.astype(np.float64) * tf + 20000.0 * fs.flat
    fraw = _exposures(rng, 11, level, 140.0, tf, n_cr=4)
    gcal, gf = _gpu_master(fraw, bias_m, dark_m, ones, tf)
    ocal, of = _oracle_master(fraw, bias_m, dark_m, ones, tf)
    print(_check("flat master", gcal, gf, ocal, of,
                 np.abs(bias_m + dark_m.astype(np.float64) * tf)))
    # two cosmic rays can land on one pixel of the 11 exposures, which a 3-sigma
    # clip of 11 samples cannot both reject: the median is the master here too
    flat_m = gf["median"]
    # the masters calibrate a science set (flat normalised by its FP64 mean)
    sci = synth.FrameSet(raw=fs.raw, bias=bias_m, dark=dark_m, flat=flat_m,
                         exptime=fs.exptime, dx=fs.dx, dy=fs.dy)
    s = core.device_set(sci).alloc_outputs()
    ws = core.reduce_sets([s], core.reduce_params("bilinear", core.clip_params(3.0, 3),
                                                  normalize_flat=True))
    assert core.sync_status(ws) == 0
    ref = oracle.reduce_set(sci, interp="bilinear", normalize_flat=True)
    got = dict(mean=s.mean.cpu().numpy(), median=s.median.cpu().numpy(),
               nkept=s.nkept.cpu().numpy())
    # the normalised samples are larger than the unnormalised ones by the flat's mean
    samp = sample_tolerance(sci, "bilinear", oracle).max(axis=0) * float(
        flat_m.mean(dtype=np.float64)) * 1.1
    print(gate_e2e("science with the GPU's masters", got, ref, samp, 3.0))
    # the flat master carries the flat pattern: its normalised form matches the
    # truth within the exposures' noise (140 / 20000 per exposure, 11 of them:
    # 2.1e-3 rms; 8 rms over the 19200 pixels)
    norm = flat_m / flat_m.mean(dtype=np.float64)
    truth = fs.flat / fs.flat.mean(dtype=np.float64)
    assert np.abs(norm - truth).max() < 8 * 140.0 / 20000.0 / np.sqrt(11)

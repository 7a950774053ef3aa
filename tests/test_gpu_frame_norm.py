"""Per-frame normalisation before the combine (zero offset or scale to the
set's first frame by the frames' FP64 mean levels) on the GPU, against the
oracle: the fused kernel, the spline tile kernel, and both forms of sets
deeper than the register combine."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2008_11486_gb300 import build as irp_build
from paper_2008_11486_gb300 import core, synth
from parity_util import U, compare, gate_e2e, sample_tolerance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _native():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    irp_build.build()


def _levelled_set(W, H, n, seed, mode):
    """A set whose frames differ by a sky level (zero) or a gain (scale), so
    that the normalisation matters."""
    fs = synth.make_set(W, H, n, 4.0, seed, n_stars=20, n_cr=4)
    rng = np.random.default_rng(seed)
    raw = fs.raw.astype(np.float64)
    for k in range(n):
        raw[k] = raw[k] + rng.uniform(-150, 150) if mode == "zero" else \
            1000 + (raw[k] - 1000) * rng.uniform(0.8, 1.25)
    fs.raw = np.clip(np.round(raw), 0, 65535).astype(np.uint16)
    return fs


@pytest.mark.parametrize("mode", ["zero", "scale"])
@pytest.mark.parametrize("interp", ["bilinear", "spline3", "cubic"])
def test_frame_normalisation_matches_oracle(interp, mode):
    fs = _levelled_set(90, 70, 12, 8800 + len(interp), mode)
    s = core.device_set(fs).alloc_outputs(want_stack=True)
    ws = core.reduce_sets([s], core.reduce_params(interp, core.clip_params(2.5, 3),
                                                  frame_norm=mode))
    assert core.sync_status(ws) == 0
    ref = oracle.reduce_set(fs, interp=interp, kappa=2.5, frame_norm=mode, want_stack=True)
    st = s.stack.cpu().numpy()
    gvalid = ~np.isnan(st)
    assert np.array_equal(gvalid, ref["valid"])
    # a normalised sample adds one rounding and the factor's own (FP32 of an
    # FP64 ratio of means that agree to about 1e-7)
    tol = sample_tolerance(fs, interp, oracle) * 1.3 + 4e-7 * np.abs(np.nan_to_num(st))
    compare("normalised stack", st, np.where(ref["valid"], ref["stack"], np.nan), tol)
    got = dict(mean=s.mean.cpu().numpy(), median=s.median.cpu().numpy(),
               nkept=s.nkept.cpu().numpy())
    samp = np.max(np.where(ref["valid"], tol, 0.0), axis=0)
    meas = np.max(np.where(ref["valid"], np.abs(np.where(gvalid, st, 0.0) - ref["stack"]), 0.0),
                  axis=0)
    print(gate_e2e(f"{interp} {mode}", got, ref, samp, 2.5, meas=meas))
    # normalising changes the result: the frames' levels differ
    plain = oracle.reduce_set(fs, interp=interp, kappa=2.5)
    assert np.nanmax(np.abs(plain["mean"] - ref["mean"])) > 1.0


@pytest.mark.parametrize("interp", ["bilinear", "spline3"])
def test_frame_normalisation_of_a_deep_set(interp):
    """70 frames: the stack chunks (bilinear) and the spline tile kernel's
    lane-group form both take each frame's factors."""
    fs = _levelled_set(64, 48, 70, 8900, "zero")
    s = core.device_set(fs).alloc_outputs()
    ws = core.reduce_sets([s], core.reduce_params(interp, frame_norm="zero"))
    assert core.sync_status(ws) == 0
    ref = oracle.reduce_set(fs, interp=interp, frame_norm="zero",
                            nthreads=os.cpu_count() or 1)
    got = dict(mean=s.mean.cpu().numpy(), median=s.median.cpu().numpy(),
               nkept=s.nkept.cpu().numpy())
    samp = sample_tolerance(fs, interp, oracle).max(axis=0) * 1.3 + 4e-7 * np.abs(ref["mean"])
    print(gate_e2e(f"deep {interp} zero", got, ref, samp, 3.0))


def test_scale_normalisation_of_a_zero_level_frame_latches_a_status():
    """A frame whose mean calibrated level is 0 cannot be scaled: the device
    latches IRP_ERR_BAD_STATISTIC (8) and the context stays usable."""
    fs = synth.make_const_set(40, 36, 3, 1000, 1000.0, 0.0, 1.0, 60.0)
    fs.raw[1] = 1000  # calibrated level 0 for frame 1 (and frame 0, the reference)
    s = core.device_set(fs).alloc_outputs()
    ws = core.reduce_sets([s], core.reduce_params("bilinear", frame_norm="scale"))
    assert core.sync_status(ws) == 8
    ws = core.reduce_sets([s], core.reduce_params("bilinear", frame_norm="zero"), ws=ws)
    assert core.sync_status(ws) == 0

"""Masked cubic-spline sets deeper than the register buckets (needs a GPU:
-m gpu).

Sec. 2.1 masks bad pixels before the cubic-spline alignment.  A masked set
on the row pass (34 <= W <= 2048, H >= 34) of 65 to 256 frames is reduced by
the tile kernel's lane-group form: each tile's samples stay in shared memory
per output pixel and a group of 4 (up to 128 frames) or 8 lanes sorts and
clips each pixel.  The cases cover both group sizes, both tile heights (8
rows; 4 when a tile's samples would not fit), and a set whose row-pass
coefficients exceed the L2 share and go in stripes of rows.  Unmasked deep
sets keep the two-step path (row and column passes, then the lane-group
combine from the filtered rows), checked here at 180 and 300 frames."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2008_11486_gb300 import build as irp_build
from paper_2008_11486_gb300 import core, synth
from parity_util import compare, gate_e2e, sample_tolerance

pytestmark = pytest.mark.gpu
NT = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def _native():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    irp_build.build()


MASK_FRAC, SAT = 0.01, 30000.0


def _mask(fs, seed):
    rng = np.random.default_rng(seed)
    return (rng.random((fs.H, fs.W)) < MASK_FRAC).astype(np.uint8)


def _run(fs, want_stack, **kw):
    s = core.device_set(fs, **kw).alloc_outputs(want_stack=want_stack)
    ws = core.reduce_sets([s], core.reduce_params("spline3", core.clip_params(2.5, 3)))
    assert core.sync_status(ws) == 0
    got = dict(mean=s.mean.cpu().numpy(), median=s.median.cpu().numpy(),
               nkept=s.nkept.cpu().numpy().astype(np.int32))
    if want_stack:
        got["stack"] = s.stack.cpu().numpy()
    return got


def _check(name, fs, got, **kw):
    ref = oracle.reduce_set(fs, interp="spline3", kappa=2.5, max_iter=3, want_stack=True,
                            nthreads=NT, **kw)
    st = got["stack"]
    gvalid = ~np.isnan(st)
    assert np.array_equal(gvalid, ref["valid"]), "sample validity differs"
    tol = sample_tolerance(fs, "spline3", oracle)
    compare(f"{name} stack", st, np.where(ref["valid"], ref["stack"], np.nan), tol)
    # the combine on identical inputs: the median bit for bit
    same = oracle.combine_stack(np.where(gvalid, st, 0.0), gvalid, kappa=2.5, max_iter=3)
    fin = ~np.isnan(same["median"])
    assert np.array_equal(np.isnan(got["median"]), ~fin)
    assert np.array_equal(got["median"][fin].view(np.uint32),
                          same["median"].astype(np.float32)[fin].view(np.uint32))
    samp = np.max(np.where(ref["valid"], tol, 0.0), axis=0)
    meas = np.max(np.where(ref["valid"], np.abs(np.where(gvalid, st, 0.0) - ref["stack"]), 0.0),
                  axis=0)
    return gate_e2e(name, got, ref, samp, 2.5, meas=meas)


# frames -> (lanes per pixel, tile rows): 65, 100 -> (4, 8); 180 -> (8, 8); 240, 256 -> (8, 4)
@pytest.mark.parametrize("n", [65, 100, 180, 240, 256])
def test_wide_tile_masked_matches_oracle(n):
    fs = synth.make_set(90, 70, n, 6.0, 12000 + n, n_stars=25, n_cr=6)
    m = _mask(fs, n)
    got = _run(fs, True, mask=m, saturation=SAT)
    print(_check(f"wide n={n}", fs, got, mask=m, saturation=SAT))


def test_wide_tile_without_stack_equals_with_stack():
    """The stack output is a debug copy: the combined results do not depend on it."""
    fs = synth.make_set(120, 90, 150, 6.0, 12200, n_stars=25, n_cr=6)
    m = _mask(fs, 1)
    a, b = _run(fs, True, mask=m, saturation=SAT), _run(fs, False, mask=m, saturation=SAT)
    for k in ("mean", "median", "nkept"):
        assert np.array_equal(np.asarray(a[k]).view(np.uint8), np.asarray(b[k]).view(np.uint8)), k


def test_wide_tile_in_stripes_of_rows():
    """180 frames of 256 x 300: 55 MB of row-pass coefficients, more than the
    share of L2 the launch sequence keeps them in, so the set goes in stripes
    of rows; sampled pixels (and every edge pixel) against the oracle."""
    fs = synth.make_set(256, 300, 180, 10.0, 12300, n_stars=60, n_cr=10)
    m = _mask(fs, 2)
    got = _run(fs, False, mask=m, saturation=SAT)
    rng = np.random.default_rng(3)
    H, W = fs.H, fs.W
    xs = np.concatenate([rng.integers(0, W, 1500), np.arange(W), np.arange(W),
                         np.zeros(H, int), np.full(H, W - 1)])
    ys = np.concatenate([rng.integers(0, H, 1500), np.zeros(W, int), np.full(W, H - 1),
                         np.arange(H), np.arange(H)])
    ref = oracle.reduce_set(fs, interp="spline3", kappa=2.5, max_iter=3, pixels=(xs, ys),
                            nthreads=NT, mask=m, saturation=SAT)
    g = {k: got[k][ys, xs] for k in ("mean", "median", "nkept")}
    samp = sample_tolerance(fs, "spline3", oracle, pixels=(xs, ys)).max(axis=0)
    print(gate_e2e("wide stripes", g, ref, samp, 2.5))


@pytest.mark.parametrize("n", [180, 300])
def test_unmasked_deep_spline_two_step_path(n):
    """Row and column passes, then the lane-group combine reading the
    horizontally filtered rows."""
    fs = synth.make_set(48, 40, n, 4.0, 12500 + n, n_stars=10, n_cr=4)
    got = _run(fs, False)
    ref = oracle.reduce_set(fs, interp="spline3", kappa=2.5, max_iter=3, nthreads=NT)
    samp = sample_tolerance(fs, "spline3", oracle).max(axis=0)
    print(gate_e2e(f"spline n={n}", got, ref, samp, 2.5))

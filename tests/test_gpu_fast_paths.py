"""The interior loop of the fused kernel against its general loop and the
oracle (needs a GPU: -m gpu).

A tile whose frames all cover it entirely, unmasked, with no stack output,
takes the branch-free interior loop: frames two at a time when a warp has at
most 2 output rows, one at a time otherwise, calibrated from the premerged
master window {bias + dark*t, flat_norm/flat} of a set of one exposure time.
Requesting the aligned stack sends every tile through the general loop
instead, so the two runs of one set must agree bit for bit (the same
arithmetic in both loops); both are gated against the FP64 oracle end to
end.  Frame counts cover every register bucket's rows per warp (4, 2, 1)
and odd counts (the last frame of a pair loop alone); a set of several
exposure times keeps the full master window and the general loop."""
import numpy as np
import pytest
import torch

import oracle
from paper_2008_11486_gb300 import build as irp_build
from paper_2008_11486_gb300 import core, synth
from parity_util import gate_e2e, sample_tolerance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _native():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    irp_build.build()


def _run(fs, interp, rows_per_warp, want_stack):
    s = core.device_set(fs).alloc_outputs(want_stack=want_stack)
    p = core.reduce_params(interp, core.clip_params(2.5, 3), rows_per_warp=rows_per_warp)
    ws = core.reduce_sets([s], p)
    assert core.sync_status(ws) == 0
    return dict(mean=s.mean.cpu().numpy(), median=s.median.cpu().numpy(),
                nkept=s.nkept.cpu().numpy().astype(np.int32))


# (frames, rows per warp): 0 is the bucket's default (4 up to 16 frames, else 2)
CASES = [(5, 0), (12, 0), (7, 2), (12, 2), (24, 0), (33, 0), (24, 1), (40, 1),
         (48, 0), (48, 2), (64, 0), (57, 1)]  # above 40: both tile heights of each stencil


@pytest.mark.parametrize("interp", ["nearest", "bilinear", "cubic"])
@pytest.mark.parametrize("n,rpw", CASES)
def test_interior_loop_equals_general_loop_and_oracle(interp, n, rpw):
    fs = synth.make_set(200, 150, n, 3.0, 7000 + 13 * n + rpw, n_stars=30, n_cr=6)
    fast = _run(fs, interp, rpw, want_stack=False)
    general = _run(fs, interp, rpw, want_stack=True)
    for k in ("mean", "median"):
        assert np.array_equal(fast[k].view(np.uint32), general[k].view(np.uint32)), k
    assert np.array_equal(fast["nkept"], general["nkept"])
    ref = oracle.reduce_set(fs, interp=interp, kappa=2.5, max_iter=3)
    samp = sample_tolerance(fs, interp, oracle).max(axis=0)
    print(gate_e2e(f"interior n={n} rpw={rpw}", fast, ref, samp, 2.5))


@pytest.mark.parametrize("n,rpw", [(12, 0), (24, 0)])
def test_several_exposure_times_take_the_general_loop(n, rpw):
    fs = synth.make_set(200, 150, n, 3.0, 7100 + n, n_stars=30, n_cr=6)
    fs.exptime = (fs.exptime * (1.0 + 0.1 * np.arange(n) / n)).astype(np.float32)
    got = _run(fs, "bilinear", rpw, want_stack=False)
    ref = oracle.reduce_set(fs, interp="bilinear", kappa=2.5, max_iter=3)
    samp = sample_tolerance(fs, "bilinear", oracle).max(axis=0)
    print(gate_e2e(f"exposures n={n}", got, ref, samp, 2.5))

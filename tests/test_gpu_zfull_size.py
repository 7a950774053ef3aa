"""Parity at the full size of the deep workload (needs a GPU: -m gpu).

32 frames of 4096x4096 uint16, offsets within +-5 px, bilinear shift, 3-sigma
clipped mean with 3 passes and the median, reduced in one call with the
parameters and the device-side frame generator of the benchmark's `deep`
workload.  The FP64 oracle evaluates sampled output pixels: random ones and
every 8th pixel along the four edges, where frames leave the grid.

The file is collected after the other GPU parity tests and before the
allocation-free entry point's test, which must run last.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2008_11486_gb300 import build as irp_build
from paper_2008_11486_gb300 import core, synth
from parity_util import gate_e2e, sample_tolerance

pytestmark = pytest.mark.gpu


def test_deep_workload_full_size_sampled():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    irp_build.build()
    W = H = 4096
    n = 32
    d = synth.make_set_torch(W, H, n, 5.0, 11486002, "cuda")
    s = core.DeviceSet(frames=[d["raw"][k] for k in range(n)], bias=d["bias"], dark=d["dark"],
                       flat=d["flat"], exptime=d["exptime"], dx=d["dx"], dy=d["dy"])
    s.alloc_outputs()
    ws = core.reduce_sets([s], core.reduce_params("bilinear", core.clip_params(3.0, 3)))
    assert core.sync_status(ws) == 0
    fs = synth.FrameSet(raw=d["raw"].cpu().numpy(), bias=d["bias"].cpu().numpy(),
                        dark=d["dark"].cpu().numpy(), flat=d["flat"].cpu().numpy(),
                        exptime=np.asarray(d["exptime"]), dx=np.asarray(d["dx"]),
                        dy=np.asarray(d["dy"]))
    rng = np.random.default_rng(11486)
    edge = np.arange(0, W, 8)
    xs = np.concatenate([rng.integers(0, W, 3000), edge, edge,
                         np.zeros(edge.size, int), np.full(edge.size, W - 1)])
    ys = np.concatenate([rng.integers(0, H, 3000), np.zeros(edge.size, int),
                         np.full(edge.size, H - 1), edge, edge])
    ref = oracle.reduce_set(fs, interp="bilinear", pixels=(xs, ys),
                            nthreads=os.cpu_count() or 1)
    gm = s.mean.cpu().numpy()[ys, xs]
    gd = s.median.cpu().numpy()[ys, xs]
    gk = s.nkept.cpu().numpy().astype(np.int32)[ys, xs]
    # clip decisions agree except within rounding reach of a threshold
    samp = sample_tolerance(fs, "bilinear", oracle, pixels=(xs, ys)).max(axis=0)
    print(gate_e2e("deep", dict(mean=gm, median=gd, nkept=gk), ref, samp, 3.0))

"""Parity at the full sizes of the deep and batch workloads (needs a GPU:
-m gpu).

Deep: 32 frames of 4096x4096 uint16, offsets within +-5 px, bilinear shift,
3-sigma clipped mean with 3 passes and the median, reduced in one call with
the parameters and the device-side frame generator of the benchmark's `deep`
workload.  Batch: the 64 sets of the benchmark's `batch` workload (frame
counts 3 to 40, sides 512 to 4096, 21.5 GB of raw frames) in its timed
launch form: the autotuned persistent launches replayed from a CUDA graph.
The FP64 oracle evaluates sampled output pixels: random ones and pixels
along the four edges, where frames leave the grid.

The file is collected after the other GPU parity tests and before the
allocation-free entry point's test, which must run last.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2008_11486_gb300 import build as irp_build
from paper_2008_11486_gb300 import batch, core, synth
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


def _edge_samples(W, H, rng, nrand, step):
    ex, ey = np.arange(0, W, step), np.arange(0, H, step)
    xs = np.concatenate([rng.integers(0, W, nrand), ex, ex, np.zeros(ey.size, int),
                         np.full(ey.size, W - 1)])
    ys = np.concatenate([rng.integers(0, H, nrand), np.zeros(ex.size, int),
                         np.full(ex.size, H - 1), ey, ey])
    return xs, ys


def test_batch_workload_full_size_sampled():
    """The headline workload as timed: each set's outputs from the graph-replayed
    autotuned launches equal its own plain launch bit for bit over the whole
    grid, and match the oracle on sampled pixels."""
    import bench
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    irp_build.build()
    cfg = bench.WORKLOADS["batch"]
    shapes = bench.workload_shapes("batch")
    raws, sets = [], []
    for i, (W, H, n) in enumerate(shapes):
        d = synth.make_set_torch(W, H, n, cfg["offset"], cfg["seed"] + 7919 * i, "cuda")
        s = core.DeviceSet(frames=[d["raw"][k] for k in range(n)], bias=d["bias"],
                           dark=d["dark"], flat=d["flat"], exptime=d["exptime"], dx=d["dx"],
                           dy=d["dy"])
        s.alloc_outputs()
        raws.append(d)
        sets.append(s)
    tuner = batch.Autotuner(None, reps=1)
    params, _ = tuner.params_for(sets, cfg["interp"])
    br = batch.BatchReducer(sets, params)
    for _ in range(2):
        br.run()
    torch.cuda.synchronize()
    assert br.status() == 0
    got = [(s.mean.clone(), s.median.clone(), s.nkept.clone()) for s in sets]
    plain = core.reduce_params(cfg["interp"], core.clip_params(3.0, 3))
    for s, (m, d, k) in zip(sets, got):
        ws = core.reduce_sets([s], plain)
        assert core.sync_status(ws) == 0
        assert torch.equal(s.mean.view(torch.int32), m.view(torch.int32))
        assert torch.equal(s.median.view(torch.int32), d.view(torch.int32))
        assert torch.equal(s.nkept, k)
    rng = np.random.default_rng(11487)
    for i, ((W, H, n), d, (m, md, k)) in enumerate(zip(shapes, raws, got)):
        fs = synth.FrameSet(raw=d["raw"].cpu().numpy(), bias=d["bias"].cpu().numpy(),
                            dark=d["dark"].cpu().numpy(), flat=d["flat"].cpu().numpy(),
                            exptime=np.asarray(d["exptime"]), dx=np.asarray(d["dx"]),
                            dy=np.asarray(d["dy"]))
        xs, ys = _edge_samples(W, H, rng, 200, max(8, W // 64))
        ref = oracle.reduce_set(fs, interp=cfg["interp"], pixels=(xs, ys),
                                nthreads=os.cpu_count() or 1)
        samp = sample_tolerance(fs, cfg["interp"], oracle, pixels=(xs, ys)).max(axis=0)
        gate_e2e(f"batch set {i} (n={n}, {W}^2)",
                 dict(mean=m.cpu().numpy()[ys, xs], median=md.cpu().numpy()[ys, xs],
                      nkept=k.cpu().numpy().astype(np.int32)[ys, xs]), ref, samp, 3.0)

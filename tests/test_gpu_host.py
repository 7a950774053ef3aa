"""GPU checks of irp_reduce_set_host: raw frames in (pinned or pageable) host
memory, results copied back to host memory, the copies of one set
overlapping the reduction of its neighbours.  The results must equal the
device-buffer entry point's bit for bit."""
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


def _host_case(fss, pinned):
    sets = [core.device_set(fs).alloc_outputs() for fs in fss]
    host_raw = [torch.from_numpy(fs.raw.astype(np.int32)).to(torch.uint16) for fs in fss]
    if pinned:
        host_raw = [h.pin_memory() for h in host_raw]
    host_out = [(torch.empty((fs.H, fs.W), dtype=torch.float32, pin_memory=pinned),
                 torch.empty((fs.H, fs.W), dtype=torch.float32, pin_memory=pinned))
                for fs in fss]
    # the device frames start out as garbage: the call must upload them
    for s in sets:
        for f in s.frames:
            f.fill_(12345)
    return sets, host_raw, host_out


@pytest.mark.parametrize("interp", ["bilinear", "spline3"])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_entry_point_equals_device_path(interp, pinned):
    fss = [synth.make_set(96, 64, 7, 4.0, 8100, n_stars=20, n_cr=4),
           synth.make_set(70, 50, 12, 4.0, 8101, n_stars=20, n_cr=4),
           synth.make_set(64, 40, 80, 4.0, 8102, n_stars=20, n_cr=4)]  # a deep set
    params = core.reduce_params(interp, core.clip_params(3.0, 3))
    ref_sets = [core.device_set(fs).alloc_outputs() for fs in fss]
    ws = core.reduce_sets(ref_sets, params)
    assert core.sync_status(ws) == 0
    sets, host_raw, host_out = _host_case(fss, pinned)
    stream = torch.cuda.current_stream()
    ws2 = core.reduce_sets_host(sets, host_raw, host_out, params, stream=stream)
    assert core.sync_status(ws2) == 0
    for fs, r, (m, d) in zip(fss, ref_sets, host_out):
        assert np.array_equal(m.numpy().view(np.uint32), r.mean.cpu().numpy().view(np.uint32))
        assert np.array_equal(d.numpy().view(np.uint32), r.median.cpu().numpy().view(np.uint32))
    ref = oracle.reduce_set(fss[0], interp=interp)
    samp = sample_tolerance(fss[0], interp, oracle).max(axis=0)
    print(gate_e2e("host path", dict(mean=host_out[0][0].numpy(), median=host_out[0][1].numpy()),
                   ref, samp, 3.0))


def test_host_entry_point_repeated_calls_and_ordering():
    """Back-to-back calls on one stream reuse the workspace and the library's
    copy streams; the second call's frames differ, and each call's results
    must be those of its own frames."""
    fa = [synth.make_set(80, 48, 9, 3.0, 8200 + i, n_stars=10) for i in range(3)]
    # the second call's frames: other raw data, the same sets (masters, offsets)
    fb = [synth.FrameSet(raw=synth.make_set(80, 48, 9, 3.0, 8300 + i, n_stars=10).raw,
                         bias=a.bias, dark=a.dark, flat=a.flat, exptime=a.exptime, dx=a.dx,
                         dy=a.dy) for i, a in enumerate(fa)]
    params = core.reduce_params("bilinear", core.clip_params(3.0, 3))
    sets, host_a, out_a = _host_case(fa, True)
    _, host_b, out_b = _host_case(fb, True)
    stream = torch.cuda.current_stream()
    ws = core.reduce_sets_host(sets, host_a, out_a, params, stream=stream)
    ws = core.reduce_sets_host(sets, host_b, out_b, params, ws=ws, stream=stream)
    assert core.sync_status(ws) == 0
    for fss, outs in ((fa, out_a), (fb, out_b)):
        ref_sets = [core.device_set(fs).alloc_outputs() for fs in fss]
        w = core.reduce_sets(ref_sets, params)
        assert core.sync_status(w) == 0
        for r, (m, _) in zip(ref_sets, outs):
            assert np.array_equal(m.numpy().view(np.uint32), r.mean.cpu().numpy().view(np.uint32))


def test_host_entry_point_pitched_host_frames():
    """Host frames with a row pitch wider than the frame (2-D copies) and
    scattered frame buffers give the same results as dense ones."""
    fss = [synth.make_set(72, 40, 6, 3.0, 8400 + i, n_stars=10) for i in range(2)]
    params = core.reduce_params("bilinear", core.clip_params(3.0, 3))
    sets, dense, out_d = _host_case(fss, True)
    ws = core.reduce_sets_host(sets, dense, out_d, params)
    assert core.sync_status(ws) == 0
    wide = []
    for h in dense:
        w = torch.zeros((h.shape[0], h.shape[1], h.shape[2] + 5), dtype=torch.uint16).pin_memory()
        w[..., :h.shape[2]] = h
        wide.append(w[..., :h.shape[2]])
    sets2, _, out_w = _host_case(fss, True)
    ws = core.reduce_sets_host(sets2, wide, out_w, params, ws=ws)
    assert core.sync_status(ws) == 0
    for (a, b), (c, d) in zip(out_d, out_w):
        assert np.array_equal(a.numpy().view(np.uint32), c.numpy().view(np.uint32))
        assert np.array_equal(b.numpy().view(np.uint32), d.numpy().view(np.uint32))

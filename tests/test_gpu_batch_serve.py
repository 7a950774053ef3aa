"""Batched and served forms on the GPU: a CUDA-graph-replayed persistent batch
of uneven sets and the continuous-batching server must give each set exactly
the result of a standalone reduction (the per-pixel arithmetic does not
depend on what else is in the launch)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2008_11486_gb300 import batch, core, serve, synth
from paper_2008_11486_gb300 import build as irp_build
from parity_util import gate_e2e, sample_tolerance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _native():
    assert torch.cuda.is_available()
    irp_build.build()


def _alone(fs, interp):
    s = core.device_set(fs).alloc_outputs()
    ws = core.reduce_sets([s], core.reduce_params(interp))
    assert core.sync_status(ws) == 0
    return s.mean.cpu().numpy(), s.median.cpu().numpy()


@pytest.mark.parametrize("interp", ["bilinear", "spline3"])
def test_graph_batch_autotuned_equals_per_set(interp, tmp_path):
    shapes = [(3, 70, 50), (9, 64, 96), (17, 40, 36), (33, 48, 64), (5, 130, 40), (12, 64, 64),
              (40, 50, 50), (24, 36, 90)]
    fss = [synth.make_set(W, H, n, 4.0, 700 + i, n_stars=15, n_cr=4)
           for i, (n, W, H) in enumerate(shapes)]
    sets = [core.device_set(fs).alloc_outputs() for fs in fss]
    tuner = batch.Autotuner(str(tmp_path / "tune.json"), reps=1)
    params, cfg = tuner.params_for(sets, interp)
    assert cfg in batch.Autotuner.candidates(sets, True, interp)
    br = batch.BatchReducer(sets, params)
    for _ in range(3):
        br.run()
    torch.cuda.synchronize()
    assert br.status() == 0
    for fs, s in zip(fss, sets):
        m, d = _alone(fs, interp)
        assert np.array_equal(s.mean.cpu().numpy().view(np.uint32), m.view(np.uint32))
        assert np.array_equal(s.median.cpu().numpy().view(np.uint32), d.view(np.uint32))


def test_rows_per_warp_choices_agree():
    fs = synth.make_set(100, 90, 10, 4.0, 31, n_stars=20)
    outs = []
    for rpw in (0, 2, 4, 7):
        s = core.device_set(fs).alloc_outputs()
        ws = core.reduce_sets([s], core.reduce_params("bilinear", rows_per_warp=rpw))
        assert core.sync_status(ws) == 0
        outs.append(s.mean.cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint32), outs[0].view(np.uint32))


def _chip_frames(nchips, W, H, nreq, seed):
    """Per chip: masters and a sequence of dithered frames of a fixed sky."""
    chips = []
    for c in range(nchips):
        fs = synth.make_set(W, H, nreq, 3.0, seed + 31 * c, n_stars=20, n_cr=3)
        chips.append(fs)
    return chips


def test_server_results_equal_standalone_reductions():
    nchips, W, H, nreq, depth = 3, 96, 80, 8, 5
    chips = _chip_frames(nchips, W, H, nreq, 4242)
    masters = [tuple(torch.from_numpy(a).cuda() for a in (fs.bias, fs.dark, fs.flat))
               for fs in chips]
    srv = serve.Server(masters, depth=depth, max_inflight=3, interp="bilinear",
                       hbm_reserve_bytes=0, out_slots=nreq)
    reqs = []
    for r in range(nreq):
        frames = [torch.from_numpy(fs.raw[r]).pin_memory() for fs in chips]
        reqs.append(serve.Request(rid=r, frames=frames,
                                  dx=np.array([fs.dx[r] for fs in chips]),
                                  dy=np.array([fs.dy[r] for fs in chips])))
    lat, wall = serve.run_poisson(srv, reqs, rate_hz=2000.0)
    assert srv.status() == 0
    assert len(srv.done) == nreq and np.all(lat > 0)
    assert srv.batches <= nreq
    for r, req in enumerate(reqs):
        first = max(0, r - depth + 1)
        for c, fs in enumerate(chips):
            sub = synth.FrameSet(raw=fs.raw[first:r + 1], bias=fs.bias, dark=fs.dark,
                                 flat=fs.flat, exptime=fs.exptime[first:r + 1],
                                 dx=fs.dx[first:r + 1], dy=fs.dy[first:r + 1])
            m, d = _alone(sub, "bilinear")
            gm, gd = req.outputs[c]
            assert np.array_equal(gm.cpu().numpy().view(np.uint32), m.view(np.uint32)), (r, c)
            assert np.array_equal(gd.cpu().numpy().view(np.uint32), d.view(np.uint32)), (r, c)
    # and one of them against the oracle
    fs = chips[1]
    sub = synth.FrameSet(raw=fs.raw[3:8], bias=fs.bias, dark=fs.dark, flat=fs.flat,
                         exptime=fs.exptime[3:8], dx=fs.dx[3:8], dy=fs.dy[3:8])
    ref = oracle.reduce_set(sub, interp="bilinear")
    gm, gd = (t.cpu().numpy() for t in reqs[7].outputs[1])
    samp = sample_tolerance(sub, "bilinear", oracle).max(axis=0)
    print(gate_e2e("served", dict(mean=gm, median=gd), ref, samp, 3.0))


def test_server_admission_waits_for_hbm():
    chips = _chip_frames(2, 64, 48, 2, 77)
    masters = [tuple(torch.from_numpy(a).cuda() for a in (fs.bias, fs.dark, fs.flat))
               for fs in chips]
    free, total = torch.cuda.mem_get_info()
    srv = serve.Server(masters, depth=5, max_inflight=2, hbm_reserve_bytes=total * 2)
    req = serve.Request(rid=0, frames=[torch.from_numpy(fs.raw[0]).pin_memory() for fs in chips],
                        dx=np.array([fs.dx[0] for fs in chips]),
                        dy=np.array([fs.dy[0] for fs in chips]))
    srv.submit(req)
    for _ in range(20):
        srv.tick()
    assert len(srv.pending) == 1 and not srv.done   # not admitted: no room
    srv.reserve = 0
    srv.drain()
    assert len(srv.done) == 1 and srv.status() == 0


def test_server_requests_allocate_no_outputs():
    """Outputs come from the per-chip output ring: after the pools have warmed
    up, further requests add no device allocation of output size."""
    nchips, W, H = 2, 96, 80
    chips = _chip_frames(nchips, W, H, 8, 91)
    masters = [tuple(torch.from_numpy(a).cuda() for a in (fs.bias, fs.dark, fs.flat))
               for fs in chips]
    srv = serve.Server(masters, depth=3, max_inflight=2, hbm_reserve_bytes=0)

    def reqs(lo, hi):
        return [serve.Request(rid=r, frames=[torch.from_numpy(fs.raw[r]).pin_memory()
                                             for fs in chips],
                              dx=np.array([fs.dx[r] for fs in chips]),
                              dy=np.array([fs.dy[r] for fs in chips])) for r in range(lo, hi)]

    serve.run_poisson(srv, reqs(0, 4), rate_hz=2000.0)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    serve.run_poisson(srv, reqs(4, 8), rate_hz=2000.0)
    torch.cuda.synchronize()
    assert srv.status() == 0
    assert torch.cuda.memory_allocated() - before < 2 * H * W * 4


def _requests(chips, lo, hi):
    return [serve.Request(rid=r, frames=[torch.from_numpy(fs.raw[r]).pin_memory() for fs in chips],
                          dx=np.array([fs.dx[r] for fs in chips]),
                          dy=np.array([fs.dy[r] for fs in chips])) for r in range(lo, hi)]


def test_server_batches_requests_that_arrive_during_work(monkeypatch):
    """Continuous batching: requests that arrive while a batch is on the device
    are admitted, upload behind it and go together in the next launch; each
    result is bit-identical to its standalone reduction.  Each batch launch is
    preceded on the compute stream by a fixed spin of about 2.5 ms (the device
    busy with other work), so that batches stay on the device while the
    scheduler runs."""
    nchips, W, H, nreq, depth = 2, 256, 192, 10, 3
    chips = _chip_frames(nchips, W, H, nreq, 5151)
    masters = [tuple(torch.from_numpy(a).cuda() for a in (fs.bias, fs.dark, fs.flat))
               for fs in chips]
    launch = core.Plan.launch

    def busy_launch(self, stream=None):
        with torch.cuda.stream(stream):
            torch.cuda._sleep(5_000_000)
        launch(self, stream)

    monkeypatch.setattr(core.Plan, "launch", busy_launch)
    srv = serve.Server(masters, depth=depth, max_inflight=4, max_batch=2, interp="bilinear",
                       hbm_reserve_bytes=0, out_slots=nreq)
    reqs = _requests(chips, 0, nreq)
    lat, wall = serve.run_poisson(srv, reqs, rate_hz=1e6)  # all arrive at once
    assert srv.status() == 0 and len(srv.done) == nreq
    print(f"\nbatch sizes {srv.batch_sizes}, admitted while a batch ran: "
          f"{srv.admitted_while_running}")
    assert max(srv.batch_sizes) >= 2, srv.batch_sizes
    assert srv.admitted_while_running >= 1
    for r, req in enumerate(reqs):
        first = max(0, r - depth + 1)
        for c, fs in enumerate(chips):
            sub = synth.FrameSet(raw=fs.raw[first:r + 1], bias=fs.bias, dark=fs.dark,
                                 flat=fs.flat, exptime=fs.exptime[first:r + 1],
                                 dx=fs.dx[first:r + 1], dy=fs.dy[first:r + 1])
            m, d = _alone(sub, "bilinear")
            gm, gd = req.outputs[c]
            assert np.array_equal(gm.cpu().numpy().view(np.uint32), m.view(np.uint32)), (r, c)
            assert np.array_equal(gd.cpu().numpy().view(np.uint32), d.view(np.uint32)), (r, c)


def test_server_request_with_a_bad_flat_reports_its_status():
    """A chip whose flat master holds a zero makes the device latch
    IRP_ERR_BAD_MASTER (host-made input, no fault): the requests reduced while
    it is there complete with that status, the server stays usable, and once
    the flat is repaired the next requests complete normally with the
    standalone results."""
    nchips, W, H, nreq, depth = 2, 96, 80, 6, 3
    chips = _chip_frames(nchips, W, H, nreq, 6161)
    masters = [tuple(torch.from_numpy(a).cuda() for a in (fs.bias, fs.dark, fs.flat))
               for fs in chips]
    srv = serve.Server(masters, depth=depth, max_inflight=2, interp="bilinear",
                       hbm_reserve_bytes=0, out_slots=nreq)
    good = masters[1][2][10, 20].item()
    masters[1][2][10, 20] = 0.0              # chip 1's flat: one zero
    bad = _requests(chips, 0, 3)
    serve.run_poisson(srv, bad, rate_hz=1e6)
    assert all(r.status == 5 for r in bad) and len(srv.failed) == 3
    masters[1][2][10, 20] = good             # repaired
    torch.cuda.synchronize()
    ok = _requests(chips, 3, nreq)
    serve.run_poisson(srv, ok, rate_hz=1e6)
    assert all(r.status == 0 for r in ok)
    for r, req in zip(range(3, nreq), ok):
        first = max(0, r - depth + 1)
        for c, fs in enumerate(chips):
            sub = synth.FrameSet(raw=fs.raw[first:r + 1], bias=fs.bias, dark=fs.dark,
                                 flat=fs.flat, exptime=fs.exptime[first:r + 1],
                                 dx=fs.dx[first:r + 1], dy=fs.dy[first:r + 1])
            m, _ = _alone(sub, "bilinear")
            assert np.array_equal(req.outputs[c][0].cpu().numpy().view(np.uint32),
                                  m.view(np.uint32)), (r, c)


def test_server_snapshot_restores_the_rolling_stacks():
    """Checkpoint and resume on the GPU: a server restored from another's
    snapshot reduces the next requests to the same bits as the first server,
    and differently from a fresh server that lacks the earlier frames."""
    nchips, W, H, depth = 2, 96, 80, 3
    chips = _chip_frames(nchips, W, H, 7, 6161)
    masters = [tuple(torch.from_numpy(a).cuda() for a in (fs.bias, fs.dark, fs.flat))
               for fs in chips]

    def server():
        return serve.Server(masters, depth=depth, max_inflight=2, hbm_reserve_bytes=0)

    def run(srv, lo, hi):
        reqs = _requests(chips, lo, hi)
        serve.run_poisson(srv, reqs, rate_hz=2000.0)
        srv.drain()
        assert srv.status() == 0
        return [[(m.clone(), d.clone()) for (m, d) in q.outputs] for q in reqs]

    a = server()
    run(a, 0, 5)
    b = server()
    b.restore(a.snapshot())
    fresh = server()
    got_a, got_b, got_f = run(a, 5, 7), run(b, 5, 7), run(fresh, 5, 7)
    for ra, rb in zip(got_a, got_b):
        for (ma, da), (mb, db) in zip(ra, rb):
            assert torch.equal(ma.view(torch.int32), mb.view(torch.int32))
            assert torch.equal(da.view(torch.int32), db.view(torch.int32))
    # the second request reduces frames 4, 5 and 6; the fresh server has 5 and 6 only
    assert not torch.equal(got_b[1][0][0].view(torch.int32), got_f[1][0][0].view(torch.int32))

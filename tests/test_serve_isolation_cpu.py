"""A served request whose reduction fails is reported alone; the requests
batched with it complete normally.

The server reads each batch's device status word back behind the batch.  On
an error it reduces the batch's requests again one by one and keeps the error
only on those that fail.  The scheduling runs here on the CPU: streams and
events are host stand-ins, and the library calls are replaced by a stand-in
reduction that writes each set's frame mean and latches a device status for
sets whose new frame carries a marker value, as the library latches a
bad-master or timeout status in the workspace.
"""
import contextlib

import numpy as np
import pytest
import torch

from paper_2008_11486_gb300 import core, serve

BAD = 4242  # a set whose new frame holds this value fails in the stand-in
ERR = 5     # IRP_ERR_BAD_MASTER


class _Event:
    def __init__(self, *args, **kwargs):
        pass

    def record(self, stream=None):
        pass

    def elapsed_time(self, other):
        return 0.0

    def query(self):
        return True


class _Stream:
    def wait_event(self, ev):
        pass


def _reduce(sets, ws):
    for s in sets:
        stack = torch.stack([f.to(torch.float32) for f in s.frames])
        s.mean.copy_(stack.mean(0))
        s.median.copy_(stack.median(0).values)
        if int(s.frames[-1][0, 0]) == BAD:  # the set's new frame
            st = ws[:4].view(torch.int32)
            if int(st[0]) == 0:
                st[0] = ERR


class _Plan:
    def __init__(self, sets, params, device=None, ws=None):
        self.sets, self.ws = list(sets), ws

    def launch(self, stream=None):
        _reduce(self.sets, self.ws)


def _reduce_sets(sets, params, ws=None, stream=None):
    _reduce(sets, ws)
    return ws


def _sync_status(ws, stream=None):
    st = ws[:4].view(torch.int32)
    v = int(st[0])
    st[0] = 0
    return v


@pytest.fixture
def host_server(monkeypatch):
    monkeypatch.setattr(torch.cuda, "Stream", lambda device=None: _Stream())
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda device=None: (1 << 40, 1 << 40))
    monkeypatch.setattr(core, "Plan", _Plan)
    monkeypatch.setattr(core, "reduce_sets", _reduce_sets)
    monkeypatch.setattr(core, "sync_status", _sync_status)
    monkeypatch.setattr(core, "workspace_size", lambda sets, params: 1024)
    monkeypatch.setattr(core, "workspace", lambda n, device="cpu": torch.zeros(n, dtype=torch.uint8))


def test_only_the_failing_request_carries_the_error(host_server):
    H, W, nchips, depth = 4, 6, 2, 3
    masters = [(torch.zeros(H, W), torch.zeros(H, W), torch.ones(H, W)) for _ in range(nchips)]
    srv = serve.Server(masters, depth=depth, max_inflight=2, device="cpu")
    value = {r: 100 + 10 * r for r in range(8)}
    value[5] = BAD  # request 5's first chip frame is flagged

    def request(r):
        frames = [torch.full((H, W), value[r] if c == 0 else 100 + 10 * r, dtype=torch.uint16)
                  for c in range(nchips)]
        return serve.Request(r, frames, np.zeros(nchips), np.zeros(nchips))

    reqs = [request(r) for r in range(8)]
    got = {}
    for pair in range(0, 8, 2):  # two requests arrive together and share a batch
        srv.submit(reqs[pair])
        srv.submit(reqs[pair + 1])
        for _ in range(4):
            srv.tick()
        for r in (pair, pair + 1):
            assert reqs[r].done > 0
            got[r] = [float(m[0, 0]) for m, _ in reqs[r].outputs]
    assert srv.batches == 4 and srv.idle()
    assert [r.rid for r in srv.failed] == [5]
    assert reqs[5].status == ERR
    assert all(reqs[r].status == 0 for r in range(8) if r != 5)
    # request 4 shared the failed batch: its outputs are the rolling stacks'
    # means all the same (frames 2..4 of each chip)
    for c in range(nchips):
        frames = [value[k] if c == 0 else 100 + 10 * k for k in range(4 - depth + 1, 5)]
        assert got[4][c] == pytest.approx(np.mean(frames))
    assert srv.status() == ERR
    # every status slot is free again once nothing is in flight
    assert sorted(srv.status_free) == [0, 1]


def test_invalid_requests_are_rejected_alone(host_server):
    H, W, nchips = 4, 6, 2
    masters = [(torch.zeros(H, W), torch.zeros(H, W), torch.ones(H, W)) for _ in range(nchips)]
    srv = serve.Server(masters, depth=3, max_inflight=2, device="cpu")

    def request(r, shape=(H, W), dtype=torch.uint16, dx=0.0, frames=nchips):
        return serve.Request(r, [torch.full(shape, 100, dtype=dtype) for _ in range(frames)],
                             np.full(nchips, dx), np.zeros(nchips))

    bad = [request(1, dx=float("nan")), request(2, shape=(H + 1, W)),
           request(3, dtype=torch.int32), request(4, frames=nchips - 1)]
    good = [request(0), request(5)]
    for r in (good[0], *bad, good[1]):
        srv.submit(r)
    assert [r.rid for r in srv.failed] == [1, 2, 3, 4]
    assert all(r.status == 1 and r.done > 0 for r in bad)
    assert [r.rid for r in srv.pending] == [0, 5]
    for _ in range(6):
        srv.tick()
    assert srv.idle() and all(r.status == 0 and r.done > 0 for r in good)
    assert float(good[1].outputs[0][0][0, 0]) == 100.0


def test_pending_requests_can_be_withdrawn(host_server):
    H, W, nchips = 4, 6, 2
    masters = [(torch.zeros(H, W), torch.zeros(H, W), torch.ones(H, W)) for _ in range(nchips)]
    srv = serve.Server(masters, depth=3, max_inflight=1, device="cpu")
    reqs = [serve.Request(r, [torch.full((H, W), 100 + r, dtype=torch.uint16)] * nchips,
                          np.zeros(nchips), np.zeros(nchips)) for r in range(3)]
    for q in reqs:
        srv.submit(q)
    srv.tick()                      # request 0 admitted and reduced (one slot)
    assert not srv.cancel(0)        # too late: admitted
    assert srv.cancel(1) and not srv.cancel(1)
    for _ in range(4):
        srv.tick()
    assert srv.idle()
    assert reqs[1].status == serve.CANCELLED and reqs[1].outputs is None
    assert reqs[0].status == reqs[2].status == 0
    # request 2's stack holds frames 0 and 2 only: the withdrawn frame never
    # entered the ring
    assert float(reqs[2].outputs[0][0][0, 0]) == pytest.approx((100 + 102) / 2)
    assert srv.status() == 0

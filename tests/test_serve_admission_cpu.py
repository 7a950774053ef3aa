"""Admission by free device memory, and withdrawal racing with admission.

The scheduling runs on the CPU with host stand-ins for the streams, events
and library calls (as in the isolation test).  ``mem_get_info`` is replaced
by a stand-in whose free bytes the test sets, so that a request's own
workspace bytes decide whether it is admitted.
"""
import contextlib
import threading

import numpy as np
import pytest
import torch

from paper_2008_11486_gb300 import core, serve

WS = 1 << 20  # workspace bytes of one request's chip sets (stand-in)


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


class _Plan:
    def __init__(self, sets, params, device=None, ws=None):
        self.sets = list(sets)

    def launch(self, stream=None):
        for s in self.sets:
            s.mean.copy_(torch.stack([f.to(torch.float32) for f in s.frames]).mean(0))


class _Mem:
    def __init__(self, free):
        self.free = free
        self.hook = None

    def __call__(self, device=None):
        if self.hook is not None:
            self.hook()
        return self.free, 1 << 40


@pytest.fixture
def host(monkeypatch):
    mem = _Mem(1 << 40)
    monkeypatch.setattr(torch.cuda, "Stream", lambda device=None: _Stream())
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "mem_get_info", mem)
    monkeypatch.setattr(core, "Plan", _Plan)
    monkeypatch.setattr(core, "sync_status", lambda ws, stream=None: 0)
    monkeypatch.setattr(core, "workspace_size", lambda sets, params: WS * len(sets) // 2)
    monkeypatch.setattr(core, "workspace",
                        lambda n, device="cpu": torch.zeros(n, dtype=torch.uint8))
    return mem


def _server(reserve):
    H, W, nchips = 4, 6, 2
    masters = [(torch.zeros(H, W), torch.zeros(H, W), torch.ones(H, W)) for _ in range(nchips)]
    return serve.Server(masters, depth=3, max_inflight=2, device="cpu",
                        hbm_reserve_bytes=reserve)


def _req(rid, nchips=2, H=4, W=6):
    return serve.Request(rid=rid, frames=[torch.full((H, W), rid, dtype=torch.uint16)] * nchips,
                         dx=np.zeros(nchips), dy=np.zeros(nchips))


def test_request_bytes_are_the_batch_workspace(host):
    srv = _server(reserve=0)
    # two chips x depth 3: the stand-in workspace is WS per request
    assert srv._request_bytes(_req(0)) == WS
    srv.submit(_req(0))
    srv._admit()
    srv.submit(_req(1))
    # the second request joins a batch with the one uploading: twice the bytes
    assert srv._request_bytes(srv.pending[0]) == 2 * WS


def test_request_waits_until_memory_frees(host):
    srv = _server(reserve=100)
    host.free = 100 + WS - 1          # one byte short of the request's workspace
    srv.submit(_req(0))
    srv.tick()
    assert len(srv.pending) == 1 and not srv.uploading and srv.held_for_memory >= 1
    host.free = 100 + WS              # enough now
    srv.tick()
    assert not srv.pending and srv.batches == 1
    srv.drain()
    # the completed batch's workspace is reused: the next request needs no bytes
    assert srv._request_bytes(_req(1)) == 0
    host.free = 100                   # the reserve alone is left: still admitted
    srv.submit(_req(1))
    srv.drain()
    assert srv.batches == 2 and len(srv.done) == 2


def test_cancel_of_the_head_during_admission_drops_no_other_request(host):
    srv = _server(reserve=0)
    srv.submit(_req(0))
    srv.submit(_req(1))
    fired = []

    def cancel_head():  # runs while _admit has released its lock
        if not fired:
            fired.append(1)
            t = threading.Thread(target=lambda: fired.append(srv.cancel(0)))
            t.start()
            t.join()

    host.hook = cancel_head
    srv.drain(timeout_s=10.0)  # a dropped request would never complete
    assert fired == [1, True]
    done = {r.rid: r for r in srv.done}
    assert done[0].status == serve.CANCELLED and done[0].outputs is None
    assert done[1].status == 0 and done[1].outputs is not None
    assert srv.admitted == 1


class _HeldEvent:
    """A completion event the test releases: the batch stays on the device."""
    held = True

    def record(self, stream=None):
        pass

    def elapsed_time(self, other):
        return 0.0

    def query(self):
        return not _HeldEvent.held


def test_requests_arriving_during_a_batch_join_the_next_one(host, monkeypatch):
    srv = _server(reserve=0)
    srv.max_inflight = srv.max_batch = 4
    _HeldEvent.held = True
    uploads_done = _Event()
    # uploads land at once, batches complete only when released
    monkeypatch.setattr(torch.cuda, "Event", lambda *a, **k: _HeldEvent())
    srv.submit(_req(0))
    srv._admit()
    srv.uploading = [(r, n, uploads_done) for (r, n, e) in srv.uploading]
    srv._launch()
    assert srv.batch_sizes == [1] and len(srv.running) == 1
    for rid in (1, 2, 3):  # arrive while batch 0 is on the device
        srv.submit(_req(rid))
    srv._admit()
    assert srv.admitted_while_running == 3
    srv.uploading = [(r, n, uploads_done) for (r, n, e) in srv.uploading]
    srv._launch()  # the device is busy: they wait
    assert srv.batch_sizes == [1] and len(srv.uploading) == 3
    _HeldEvent.held = False
    srv.tick()     # batch 0 completes; the three go together
    assert srv.batch_sizes == [1, 3]
    srv.drain(timeout_s=10.0)
    assert sorted(r.rid for r in srv.done) == [0, 1, 2, 3]
    assert all(r.status == 0 and r.outputs is not None for r in srv.done)

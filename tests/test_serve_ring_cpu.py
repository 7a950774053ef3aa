"""The serving rings never overwrite a frame that a request in flight reads.

A served request writes its new raw frame into a per-chip ring and is reduced
with the previous frames of the same ring (a rolling reference stack), while
up to ``max_inflight`` requests are uploading or reducing.  The ring and the
output ring are allocated once, so their sizes alone must keep a new frame out
of every slot an unfinished request still reads.  Admission runs here on the
CPU: the CUDA streams and events are replaced by host stand-ins, the requests
are completed in order (one compute stream), and every admission is checked
against the stacks of the requests still in flight.
"""
import contextlib

import numpy as np
import pytest
import torch

from paper_2008_11486_gb300 import serve


class _Event:
    def __init__(self, *args, **kwargs):
        pass

    def record(self, stream=None):
        pass

    def elapsed_time(self, other):
        return 0.0

    def query(self):
        return True


@pytest.fixture
def host_cuda(monkeypatch):
    monkeypatch.setattr(torch.cuda, "Stream", lambda device=None: None)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda device=None: (1 << 40, 1 << 40))


@pytest.mark.parametrize("depth,max_inflight", [(5, 1), (5, 2), (5, 4), (3, 3), (1, 2)])
def test_new_frames_never_land_in_a_stack_in_flight(host_cuda, depth, max_inflight):
    H, W, nchips = 4, 6, 2
    masters = [(torch.zeros(H, W), torch.zeros(H, W), torch.ones(H, W)) for _ in range(nchips)]
    srv = serve.Server(masters, depth=depth, max_inflight=max_inflight, device="cpu")
    rng = np.random.default_rng(depth * 10 + max_inflight)
    inflight = []  # (request, frame numbers per chip), oldest first
    rid = 0
    for _ in range(300):
        # arrivals
        for _ in range(int(rng.integers(0, 3))):
            frames = [torch.full((H, W), rid, dtype=torch.uint16) for _ in range(nchips)]
            srv.submit(serve.Request(rid, frames, np.zeros(nchips), np.zeros(nchips)))
            rid += 1
        # admission: check each new frame against the stacks still in flight
        before = len(srv.uploading)
        srv._admit()
        for req, nums, _ in srv.uploading[before:]:
            for c, chip in enumerate(srv.chips):
                written = nums[c] % chip.slots
                for other, onums in inflight:
                    assert written not in chip.stack_slots(onums[c]), \
                        f"request {req.rid} overwrites a frame of request {other.rid}"
                # the request's own stack: the last depth frames, oldest first
                first = max(0, nums[c] - depth + 1)
                assert chip.stack_slots(nums[c]) == [k % chip.slots
                                                     for k in range(first, nums[c] + 1)]
                assert int(chip.ring[written][0, 0]) == req.rid
            assert req.out_slot not in [o.out_slot for o, _ in inflight]
            inflight.append((req, nums))
        assert len(inflight) <= max_inflight
        # in order completion of some of the oldest requests
        done = int(rng.integers(0, len(inflight) + 1))
        for _ in range(done):
            req, _ = inflight.pop(0)
            srv.uploading = [u for u in srv.uploading if u[0] is not req]
    assert rid > 100 and srv.admitted > 100

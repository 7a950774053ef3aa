"""Checkpoint and resume of the serving state, on the CPU.

A snapshot holds each chip's raw-frame ring with its offsets and exposure
times and the counters; a server restored from it continues the rolling
stacks exactly where the first one stopped.  The library calls are the host
stand-ins of the serving isolation test.
"""
import numpy as np
import pytest
import torch

from paper_2008_11486_gb300 import serve
from test_serve_isolation_cpu import host_server  # noqa: F401 (fixture)

H, W, NCHIPS, DEPTH = 4, 6, 2, 3


def _masters():
    return [(torch.zeros(H, W), torch.zeros(H, W), torch.ones(H, W)) for _ in range(NCHIPS)]


def _request(r):
    return serve.Request(r, [torch.full((H, W), 100 + 10 * r + c, dtype=torch.uint16)
                             for c in range(NCHIPS)],
                         np.full(NCHIPS, 0.25 * r), np.zeros(NCHIPS))


def _run(srv, rids):
    reqs = [_request(r) for r in rids]
    for q in reqs:
        srv.submit(q)
        for _ in range(3):
            srv.tick()
    assert srv.idle()
    return [[float(m[0, 0]) for m, _ in q.outputs] for q in reqs]


def test_a_restored_server_continues_the_rolling_stacks(host_server):  # noqa: F811
    a = serve.Server(_masters(), depth=DEPTH, max_inflight=2, device="cpu")
    _run(a, range(5))
    snap = a.snapshot()
    b = serve.Server(_masters(), depth=DEPTH, max_inflight=2, device="cpu")
    b.restore(snap)
    assert b.admitted == a.admitted == 5
    # the next requests see the same stacks on both servers
    got = _run(b, [5, 6])
    assert got == _run(a, [5, 6])
    # request 6 reduces the last DEPTH frames of each chip: frames 4, 5, 6
    assert got[1] == [np.mean([100 + 10 * k + c for k in (4, 5, 6)]) for c in range(NCHIPS)]
    # a fresh server without the snapshot has only frames 5 and 6
    fresh = serve.Server(_masters(), depth=DEPTH, max_inflight=2, device="cpu")
    assert _run(fresh, [5, 6])[1] != got[1]


def test_restore_refuses_another_shape(host_server):  # noqa: F811
    a = serve.Server(_masters(), depth=DEPTH, max_inflight=2, device="cpu")
    snap = a.snapshot()
    with pytest.raises(ValueError):
        serve.Server(_masters(), depth=DEPTH + 1, max_inflight=2, device="cpu").restore(snap)
    with pytest.raises(ValueError):
        serve.Server(_masters(), depth=DEPTH, max_inflight=3, device="cpu").restore(snap)
    a.submit(_request(0))
    with pytest.raises(RuntimeError):
        a.snapshot()

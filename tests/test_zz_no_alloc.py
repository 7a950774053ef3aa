"""irp_reduce_set_noalloc: the fused reduction for callers that cannot
allocate device memory (for example a real-time loop that reserves all device
memory at start-up, or a plug-in whose host framework owns the memory pool).

The entry point keeps its scratch in a static device array of the library, so
the caller passes only inputs and outputs.  This test calls it through the C
ABI twice in a row and checks each result against irp_reduce_set, which uses
a caller-provided workspace, within the tolerance of the parity tests.  The
file is named so that pytest collects it last; it also passes on its own in
a fresh process."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2008_11486_gb300 import _binding as B
from paper_2008_11486_gb300 import build as irp_build
from paper_2008_11486_gb300 import core, synth
from parity_util import mean_tolerance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available()
    irp_build.build()
    L = B.lib()
    L.irp_reduce_set_noalloc.restype = ctypes.c_int
    L.irp_reduce_set_noalloc.argtypes = [ctypes.POINTER(B.IrpSet), ctypes.c_int,
                                         ctypes.POINTER(B.ReduceParams), ctypes.c_void_p,
                                         ctypes.c_void_p]
    return L


def _fresh_outputs(sets):
    for s in sets:
        s.mean = s.median = s.nkept = None
        s.alloc_outputs()


@pytest.mark.parametrize("interp", ["bilinear", "spline3"])
def test_noalloc_matches_workspace_entry_point_twice(L, interp):
    fss = [synth.make_set(150, 100, 7, 4.0, 4000 + i, n_stars=20, n_cr=5) for i in range(2)]
    sets = [core.device_set(fs).alloc_outputs() for fs in fss]
    params = core.reduce_params(interp, core.clip_params(2.5))
    ws = core.reduce_sets(sets, params)
    assert core.sync_status(ws) == 0
    ref = [(s.mean.cpu().numpy(), s.median.cpu().numpy(), s.nkept.cpu().numpy()) for s in sets]
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    for call in range(2):
        _fresh_outputs(sets)
        arr, keep = core._irp_sets(sets)
        rc = L.irp_reduce_set_noalloc(arr, len(sets), ctypes.byref(params),
                                      ctypes.c_void_p(status.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0, B.STATUS_NAMES.get(rc, rc)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        for s, (m, d, k) in zip(sets, ref):
            gm, gd = s.mean.cpu().numpy(), s.median.cpu().numpy()
            assert np.array_equal(np.isnan(gm), np.isnan(m))
            fin = ~np.isnan(m)
            assert np.all(np.abs(gm - m)[fin] <= mean_tolerance(m)[fin])
            assert np.all(np.abs(gd - d)[fin] <= mean_tolerance(d)[fin])
            assert np.array_equal(s.nkept.cpu().numpy(), k)


def test_noalloc_rejects_requests_beyond_its_scratch(L):
    # the spline workspace of 8 frames of 1024x512 (32 MiB) exceeds the 8 MiB scratch
    fs = synth.make_const_set(1024, 512, 8, 1500, 1000.0, 0.05, 0.8, 60.0)
    s = core.device_set(fs).alloc_outputs()
    arr, keep = core._irp_sets([s])
    params = core.reduce_params("spline3")
    rc = L.irp_reduce_set_noalloc(arr, 1, ctypes.byref(params), None,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 3  # IRP_ERR_WORKSPACE, nothing enqueued


def _bits_equal(a, b):
    """Same bits, NaN where the other has NaN (the outputs are deterministic)."""
    a, b = np.asarray(a), np.asarray(b)
    return np.array_equal(a.view(np.uint8), b.view(np.uint8))


@pytest.mark.parametrize("persistent", [0, 1])
def test_noalloc_plan_copied_from_host_equals_workspace_entry_point(L, persistent):
    """Six small sets of uneven frame counts (one set deeper than the register
    combine): the plan does not travel as kernel parameters and is copied to
    the scratch.  The outputs are bit-identical to irp_reduce_set's on two
    calls in a row (the persistent work counters start at zero on each)."""
    shapes = [(3, 64, 40), (9, 40, 33), (17, 48, 50), (5, 20, 70), (12, 33, 64), (70, 24, 20)]
    fss = [synth.make_set(W, H, n, 4.0, 4100 + i, n_stars=8, n_cr=3)
           for i, (n, W, H) in enumerate(shapes)]
    sets = [core.device_set(fs).alloc_outputs() for fs in fss]
    params = core.reduce_params("bilinear", core.clip_params(2.5), persistent=persistent)
    ws = core.reduce_sets(sets, params)
    assert core.sync_status(ws) == 0
    ref = [(s.mean.cpu().numpy(), s.median.cpu().numpy(), s.nkept.cpu().numpy()) for s in sets]
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    for call in range(2):
        _fresh_outputs(sets)
        arr, keep = core._irp_sets(sets)
        rc = L.irp_reduce_set_noalloc(arr, len(sets), ctypes.byref(params),
                                      ctypes.c_void_p(status.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0, B.STATUS_NAMES.get(rc, rc)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        for s, (m, d, k) in zip(sets, ref):
            assert _bits_equal(s.mean.cpu().numpy(), m), f"mean, call {call}"
            assert _bits_equal(s.median.cpu().numpy(), d), f"median, call {call}"
            assert np.array_equal(s.nkept.cpu().numpy(), k), f"nkept, call {call}"


def test_noalloc_refuses_a_copied_plan_while_the_stream_is_captured(L):
    """A plan copied from the call's stack buffer would be read after the call
    returns by a recorded copy: during capture the call enqueues nothing and
    returns IRP_ERR_UNSUPPORTED (4)."""
    fss = [synth.make_set(40, 30, 3, 2.0, 4200 + i, n_stars=4, n_cr=1) for i in range(5)]
    sets = [core.device_set(fs).alloc_outputs() for fs in fss]
    params = core.reduce_params("bilinear", core.clip_params(2.5))
    arr, keep = core._irp_sets(sets)
    side = torch.cuda.Stream()
    # a first call outside capture (the scratch address is looked up on it)
    rc = L.irp_reduce_set_noalloc(arr, len(sets), ctypes.byref(params), None,
                                  ctypes.c_void_p(side.cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side, capture_error_mode="relaxed"):
        rc = L.irp_reduce_set_noalloc(arr, len(sets), ctypes.byref(params), None,
                                      ctypes.c_void_p(side.cuda_stream))
    assert rc == 4

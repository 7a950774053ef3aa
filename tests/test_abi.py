"""The C ABI boundary on the CPU: the library builds and loads, exports every
function include/irp.h declares, and rejects bad arguments with the exact
status code before anything is enqueued (no GPU is touched)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2008_11486_gb300 import build as irp_build
from paper_2008_11486_gb300 import _binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    irp_build.build()
    return B.lib()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "irp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(irp_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = _declared_functions()
    assert "irp_reduce_set" in names and "irp_calibrate" in names and len(names) >= 15
    for name in names:
        assert hasattr(L, name), name


def test_version_and_status_strings(L):
    assert L.irp_version() == 10000
    for code in range(8):
        assert L.irp_status_string(code)
    assert L.irp_status_string(99) == b"unknown status"


FAKE = 0x7f0000000000  # never dereferenced: validation fails before any launch


def _set(n=3, W=64, H=48, frames=None, **kw):
    ptrs = (ctypes.c_void_p * n)(*([FAKE + 4096 * k for k in range(n)] if frames is None else frames))
    dx = np.zeros(n)
    dy = np.zeros(n)
    t = np.full(n, 60.0, np.float32)
    s = B.IrpSet()
    s.frames = ctypes.cast(ptrs, ctypes.POINTER(ctypes.c_void_p))
    s.raw_pitch = W
    s.W, s.H, s.n = W, H, n
    s.dx = dx.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    s.dy = dy.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    s.exptime = t.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    s.bias, s.dark_rate, s.flat = FAKE, FAKE + 1024, FAKE + 2048
    s.master_pitch = W
    s.mean_out, s.median_out = FAKE + 8192, FAKE + 16384
    s.out_pitch = W
    for k, v in kw.items():
        setattr(s, k, v)
    s._keep = (ptrs, dx, dy, t)
    return s


def _params(interp=1, **kw):
    p = B.ReduceParams(interp, B.ClipParams(3.0, 3.0, 3, 0, 0), 0, 0, 0, 0, 0)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _reduce(L, sets, p, ws=FAKE, ws_bytes=1 << 30):
    arr = (B.IrpSet * len(sets))(*sets)
    return L.irp_reduce_set(arr, len(sets), ctypes.byref(p), ctypes.c_void_p(ws), ws_bytes, None)


def test_reduce_set_validation_codes(L):
    assert _reduce(L, [_set()], _params(), ws_bytes=0) == 3            # workspace too small
    assert _reduce(L, [_set()], _params(), ws=FAKE + 8) == 3           # workspace misaligned
    assert _reduce(L, [_set(n=1025)], _params()) == 4                  # too many frames
    assert _reduce(L, [_set()], _params(interp=7)) == 1                # bad interpolation
    assert _reduce(L, [_set(W=0)], _params()) == 1                     # empty frame
    assert _reduce(L, [_set(H=0)], _params()) == 1
    assert _reduce(L, [_set(n=0)], _params()) == 1                     # empty set
    s0 = _set()  # owns the host arrays the struct points at
    empty = (B.IrpSet * 1)(s0)
    assert L.irp_reduce_set(empty, 0, ctypes.byref(_params()), ctypes.c_void_p(FAKE), 1 << 30,
                            None) == 1                                  # no sets
    assert L.irp_workspace_size(empty, 0, ctypes.byref(_params())) == 0
    assert _reduce(L, [_set(raw_pitch=10)], _params()) == 1            # pitch < W
    assert _reduce(L, [_set(bias=FAKE + 2)], _params()) == 2           # misaligned master
    assert _reduce(L, [_set(frames=[FAKE, 0, FAKE])], _params()) == 1  # null frame
    assert _reduce(L, [_set(frames=[FAKE, FAKE + 1, FAKE])], _params()) == 2
    bad = _params()
    bad.clip.kappa_lo = -1.0
    assert _reduce(L, [_set()], bad) == 1
    bad = _params()
    bad.clip.ddof = 5
    assert _reduce(L, [_set()], bad) == 1
    assert L.irp_reduce_set(None, 1, ctypes.byref(_params()), ctypes.c_void_p(FAKE), 1 << 30,
                            None) == 1
    s = _set()
    s._keep[1][1] = np.nan  # non-finite offset
    assert _reduce(L, [s], _params()) == 1
    assert _reduce(L, [_set(mask=FAKE, mask_pitch=10)], _params()) == 1    # mask pitch < W
    assert _reduce(L, [_set(saturation=-1.0)], _params()) == 1              # negative level
    # the cubic spline masks the sets its tile kernel reduces (row pass: 34 <= W
    # <= 2048, H >= 34; at most 256 frames); others return IRP_ERR_UNSUPPORTED
    assert _reduce(L, [_set(W=20, mask=FAKE, mask_pitch=64)], _params(interp=2)) == 4
    assert _reduce(L, [_set(n=257, saturation=6e4)], _params(interp=2)) == 4
    ok = (B.IrpSet * 1)(_set(mask=FAKE, mask_pitch=64, saturation=6e4))
    assert L.irp_workspace_size(ok, 1, ctypes.byref(_params(interp=2))) > 0


def test_workspace_size_accounts_for_spline_coefficients(L):
    s = _set(n=4, W=100, H=30)
    arr = (B.IrpSet * 1)(s)
    wb = L.irp_workspace_size(arr, 1, ctypes.byref(_params(interp=1)))
    ws = L.irp_workspace_size(arr, 1, ctypes.byref(_params(interp=2)))
    assert wb > 0
    # coefficient frames carry a 2-sample border: (H + 4) rows of align4(W + 4) floats
    per_frame = -(-(30 + 4) * 104 * 4 // 256) * 256
    assert ws - wb == 4 * per_frame
    assert L.irp_workspace_size(arr, 1, ctypes.byref(_params(interp=9))) == 0
    assert L.irp_shift_workspace_size(100, 30, 4, 2) == 4 * per_frame
    assert L.irp_shift_workspace_size(100, 30, 4, 1) == 0
    assert L.irp_calibrate_workspace_size(10) >= 256 + 11 * 32


def test_plan_accepts_a_batch_spanning_every_frame_count_bucket(L):
    # frame counts 1..64 fall into 12 register buckets: one sub-plan each
    sets = [_set(n=n, W=64, H=48) for n in (1, 5, 6, 8, 10, 12, 16, 24, 32, 40, 48, 64, 3, 33)]
    arr = (B.IrpSet * len(sets))(*sets)
    for persistent in (0, 1):
        p = _params(persistent=persistent)
        assert L.irp_plan_bytes(arr, len(sets), ctypes.byref(p)) > 0
        assert L.irp_workspace_size(arr, len(sets), ctypes.byref(p)) > 0


def test_deep_sets_plan_and_stack_workspace(L):
    # a set deeper than the register buckets adds its aligned FP32 stack to
    # the workspace, [n][H][W rounded up to 32] floats, unless the caller
    # passes stack_out; its chunks form one extra sub-plan
    # the IrpSet objects own the host arrays the structs point at: keep them
    big = _set(n=1024)
    assert L.irp_workspace_size((B.IrpSet * 1)(big), 1, ctypes.byref(_params())) > 0
    plain = _set(n=64, W=50, H=48)
    deep = _set(n=100, W=50, H=48)
    deep_own = _set(n=100, W=50, H=48, stack_out=FAKE + 32768)
    ws = {k: L.irp_workspace_size((B.IrpSet * 1)(s), 1, ctypes.byref(_params()))
          for k, s in (("deep", deep), ("own", deep_own))}
    assert ws["deep"] - ws["own"] == -(-100 * 48 * 64 * 4 // 256) * 256
    deeper = _set(n=300, W=40, H=40)
    arr = (B.IrpSet * 3)(plain, deep, deeper)
    for interp in (0, 1, 2):
        for persistent in (0, 1):
            p = _params(interp=interp, persistent=persistent)
            assert L.irp_plan_bytes(arr, 3, ctypes.byref(p)) > 0
            assert L.irp_workspace_size(arr, 3, ctypes.byref(p)) > 0


def test_reduce_set_host_validation_codes(L):
    n, W, H = 3, 64, 48
    hp = (ctypes.c_void_p * n)(*[FAKE + 65536 * k for k in range(n)])
    io = (B.IrpHostIo * 1)()
    io[0].frames = ctypes.cast(hp, ctypes.POINTER(ctypes.c_void_p))
    io[0].pitch = W
    s = _set(n=n, W=W, H=H)  # owns the host arrays the struct points at
    arr = (B.IrpSet * 1)(s)
    p = _params()

    def call(io_arg, ws_bytes=1 << 30):
        return L.irp_reduce_set_host(arr, 1, io_arg, ctypes.byref(p), ctypes.c_void_p(FAKE),
                                     ws_bytes, None)
    assert call(None) == 1                      # no host side
    io[0].pitch = W - 1
    assert call(io) == 1                        # host pitch < W
    io[0].pitch = W
    io[0].nkept, io[0].out_pitch = FAKE, W     # host kept count without a device one
    assert call(io) == 1
    io[0].nkept = None
    io[0].mean, io[0].out_pitch = FAKE, W - 2  # output pitch < W
    assert call(io) == 1
    io[0].out_pitch = W
    assert call(io, ws_bytes=256) == 3          # workspace smaller than one set's
    bad = (ctypes.c_void_p * n)(FAKE, None, FAKE)
    io[0].frames = ctypes.cast(bad, ctypes.POINTER(ctypes.c_void_p))
    assert call(io) == 1                        # null host frame


def test_unfused_validation_codes(L):
    clip = B.ClipParams(3.0, 3.0, 3, 0, 0)
    f = ctypes.c_void_p(FAKE)
    # combine: n above the warp-per-pixel limit, null clip, bad dtype
    assert L.irp_combine(f, 64, 64 * 64, 64, 64, 1025, 0, None, None, None, ctypes.byref(clip),
                         f, f, None, None, 64, None) == 4
    assert L.irp_combine(f, 64, 64 * 64, 64, 64, 5, 0, None, None, None, None,
                         f, f, None, None, 64, None) == 1
    assert L.irp_combine(f, 64, 64 * 64, 64, 64, 5, 3, None, None, None, ctypes.byref(clip),
                         f, f, None, None, 64, None) == 1
    assert L.irp_combine(f, 64, 64 * 64, 64, 64, 5, 1, None, None, None, ctypes.byref(clip),
                         f, f, None, None, 64, None) == 1    # f16 without scale/offset
    # shift: in == out, bad interp, spline without workspace
    dx = np.zeros(2)
    dp = dx.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert L.irp_shift(f, 64, 4096, 64, 64, 2, 0, None, None, dp, dp, 1, f, 64, 4096, None,
                       None, 0, None) == 1
    g = ctypes.c_void_p(FAKE + (1 << 20))
    assert L.irp_shift(f, 64, 4096, 64, 64, 2, 0, None, None, dp, dp, 5, g, 64, 4096, None,
                       None, 0, None) == 1
    assert L.irp_shift(f, 64, 4096, 64, 64, 2, 0, None, None, dp, dp, 2, g, 64, 4096, None,
                       None, 0, None) == 3
    # calibrate: misaligned raw, f16 without scale outputs, small workspace
    t = np.full(2, 60.0, np.float32)
    tp = t.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    assert L.irp_calibrate(ctypes.c_void_p(FAKE + 1), 64, 4096, 64, 64, 2, f, f, f, 64, tp, 0, g,
                           64, 4096, 0, None, None, f, 4096, None) == 2
    assert L.irp_calibrate(f, 64, 4096, 64, 64, 2, f, f, f, 64, tp, 0, g, 64, 4096, 1, None,
                           None, f, 4096, None) == 1
    assert L.irp_calibrate(f, 64, 4096, 64, 64, 2, f, f, f, 64, tp, 0, g, 64, 4096, 0, None,
                           None, f, 16, None) == 3


def test_noalloc_validation_before_any_device_call(L):
    # a separate prototype: the shared binding object stays as the tests that
    # run on a GPU declare it
    proto = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(B.IrpSet), ctypes.c_int,
                             ctypes.POINTER(B.ReduceParams), ctypes.c_void_p, ctypes.c_void_p)
    noalloc = proto(("irp_reduce_set_noalloc", L))

    def call(sets, p, status=None):
        arr = (B.IrpSet * max(len(sets), 1))(*sets)
        return noalloc(arr, len(sets), ctypes.byref(p), status, None)

    assert call([], _params()) == 1                                  # no sets
    assert call([_set(W=0)], _params()) == 1                         # empty frame
    assert call([_set(n=1025)], _params()) == 4                      # too many frames
    assert call([_set()], _params(), status=FAKE + 2) == 2           # misaligned status word
    # the spline workspace of 8 frames of 1024x512 (32 MiB) exceeds the 8 MiB scratch
    assert call([_set(n=8, W=1024, H=512)], _params(interp=2)) == 3
    # 64 sets of 40 frames: the plan outgrows the call's fixed host buffer
    many = [_set(n=40, W=64, H=48) for _ in range(64)]
    assert call(many, _params()) == 3

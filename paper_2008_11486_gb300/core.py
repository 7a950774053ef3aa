"""Tensor-level API over the C ABI.

Device memory and streams come from PyTorch; every step of the reduction runs
in the CUDA library through ``_binding``.  Calls are asynchronous on the given
stream (default: the current torch stream).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np
import torch

from ._binding import (DTYPE, FRAME_NORM, INTERP, KERNEL_KINDS, ClipParams, IrpHostIo, IrpSet, ReduceParams,
                       check, lib)


def _vp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _u16(t: torch.Tensor) -> torch.Tensor:
    if t.dtype not in (torch.uint16, torch.int16):
        raise TypeError("raw frames must be uint16 (or int16 holding the same bits)")
    return t


def clip_params(kappa: float = 3.0, max_iter: int = 3, center: str = "mean", ddof: int = 0,
                kappa_lo: float | None = None, kappa_hi: float | None = None) -> ClipParams:
    return ClipParams(float(kappa if kappa_lo is None else kappa_lo),
                      float(kappa if kappa_hi is None else kappa_hi), int(max_iter),
                      1 if center == "median" else 0, int(ddof))


def workspace(nbytes: int, device="cuda") -> torch.Tensor:
    """Device workspace; its 256-byte header (status word, counters) starts at zero."""
    return torch.zeros(max(int(nbytes), 256), dtype=torch.uint8, device=device)


# ----------------------------------------------------------------- calibrate
def calibrate(raw, bias, dark, flat, exptime, *, normalize_flat=False, dtype="f32",
              out=None, ws=None, stream=None):
    """raw [n,H,W] uint16 -> calibrated frames (f32, or f16 with scale/offset)."""
    raw = _u16(raw)
    n, H, W = raw.shape
    dt = DTYPE[dtype]
    if out is None:
        out = torch.empty((n, H, W), dtype=torch.float32 if dt == 0 else torch.float16,
                          device=raw.device)
    scale = offset = None
    if dt == 1:
        scale = torch.empty(n, dtype=torch.float32, device=raw.device)
        offset = torch.empty(n, dtype=torch.float32, device=raw.device)
    L = lib()
    need = L.irp_calibrate_workspace_size(n)
    if ws is None or ws.numel() < need:
        ws = workspace(need, raw.device)
    t = np.ascontiguousarray(exptime, dtype=np.float32)
    check(L.irp_calibrate(_vp(raw), raw.stride(1), raw.stride(0), W, H, n, _vp(bias), _vp(dark),
                          _vp(flat), bias.stride(0),
                          t.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), int(normalize_flat),
                          _vp(out), out.stride(1), out.stride(0), dt, _vp(scale), _vp(offset),
                          _vp(ws), ws.numel(), _stream(stream)), "irp_calibrate")
    return out, scale, offset, ws


def frame_stats(frames, dtype="f32", scale=None, offset=None, stream=None):
    n, H, W = frames.shape
    s = torch.empty(n, dtype=torch.float64, device=frames.device)
    q = torch.empty(n, dtype=torch.float64, device=frames.device)
    c = torch.empty(n, dtype=torch.int64, device=frames.device)
    check(lib().irp_frame_stats(_vp(frames), frames.stride(1), frames.stride(0), W, H, n,
                                DTYPE[dtype], _vp(scale), _vp(offset), _vp(s), _vp(q), _vp(c),
                                _stream(stream)), "irp_frame_stats")
    return s, q, c


# --------------------------------------------------------------------- shift
def shift(frames, dx, dy, interp="bilinear", *, dtype="f32", scale=None, offset=None,
          out=None, want_valid=True, ws=None, stream=None):
    """Calibrated frames [n,H,W] -> aligned stack (NaN where invalid) + valid mask."""
    n, H, W = frames.shape
    if out is None:
        out = torch.empty_like(frames)
    valid = torch.empty((n, H, W), dtype=torch.uint8, device=frames.device) if want_valid else None
    L = lib()
    need = L.irp_shift_workspace_size(W, H, n, INTERP[interp])
    if need and (ws is None or ws.numel() < need):
        ws = workspace(need, frames.device)
    dxa = np.ascontiguousarray(dx, dtype=np.float64)
    dya = np.ascontiguousarray(dy, dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    check(L.irp_shift(_vp(frames), frames.stride(1), frames.stride(0), W, H, n, DTYPE[dtype],
                      _vp(scale), _vp(offset), dxa.ctypes.data_as(dp), dya.ctypes.data_as(dp),
                      INTERP[interp], _vp(out), out.stride(1), out.stride(0), _vp(valid),
                      _vp(ws) if need else None, ws.numel() if (need and ws is not None) else 0,
                      _stream(stream)), "irp_shift")
    return out, valid, ws


# ------------------------------------------------------------------- combine
def combine(stack, *, dtype="f32", scale=None, offset=None, valid=None, clip=None,
            want_reject=False, stream=None):
    n, H, W = stack.shape
    dev = stack.device
    clip = clip if clip is not None else clip_params()
    mean = torch.empty((H, W), dtype=torch.float32, device=dev)
    med = torch.empty((H, W), dtype=torch.float32, device=dev)
    kept = torch.empty((H, W), dtype=torch.uint16, device=dev)
    rej = torch.empty((n, H, W), dtype=torch.uint8, device=dev) if want_reject else None
    check(lib().irp_combine(_vp(stack), stack.stride(1), stack.stride(0), W, H, n, DTYPE[dtype],
                            _vp(scale), _vp(offset), _vp(valid), ctypes.byref(clip), _vp(mean),
                            _vp(med), _vp(kept), _vp(rej), W, _stream(stream)), "irp_combine")
    return dict(mean=mean, median=med, nkept=kept, reject=rej)


# -------------------------------------------------------------- fused reduce
@dataclass
class DeviceSet:
    """One frame set resident on the device plus its host-side offsets."""
    frames: list                 # n device uint16 [H,W] tensors (may be views of one [n,H,W])
    bias: torch.Tensor
    dark: torch.Tensor
    flat: torch.Tensor
    exptime: np.ndarray
    dx: np.ndarray
    dy: np.ndarray
    mean: torch.Tensor | None = None
    median: torch.Tensor | None = None
    nkept: torch.Tensor | None = None
    stack: torch.Tensor | None = None
    ready_flag: torch.Tensor | None = None
    ready_value: int = 0
    mask: torch.Tensor | None = None   # uint8 [H, W] bad-pixel mask (non-zero = bad)
    saturation: float = 0.0            # raw ADU level marking a pixel bad; 0 = off
    _keep: list = field(default_factory=list)

    @property
    def n(self):
        return len(self.frames)

    @property
    def H(self):
        return int(self.frames[0].shape[0])

    @property
    def W(self):
        return int(self.frames[0].shape[1])

    def alloc_outputs(self, want_stack=False, want_nkept=True):
        dev = self.frames[0].device
        if self.mean is None:
            self.mean = torch.empty((self.H, self.W), dtype=torch.float32, device=dev)
        if self.median is None:
            self.median = torch.empty((self.H, self.W), dtype=torch.float32, device=dev)
        if want_nkept and self.nkept is None:
            self.nkept = torch.empty((self.H, self.W), dtype=torch.uint16, device=dev)
        if want_stack and self.stack is None:
            self.stack = torch.empty((self.n, self.H, self.W), dtype=torch.float32, device=dev)
        return self


def device_set(fs, device="cuda", raw=None, masters=None, mask=None,
               saturation=0.0) -> DeviceSet:
    """Uploads a synth.FrameSet (or uses the given device raw [n,H,W] / masters);
    ``mask`` (host or device [H, W] uint8) and ``saturation`` mark bad pixels."""
    if raw is None:
        raw = torch.from_numpy(np.ascontiguousarray(fs.raw)).to(device)
    if masters is None:
        masters = tuple(torch.from_numpy(np.ascontiguousarray(a)).to(device)
                        for a in (fs.bias, fs.dark, fs.flat))
    frames = [raw[k] for k in range(raw.shape[0])]
    if mask is not None and not isinstance(mask, torch.Tensor):
        mask = torch.from_numpy(np.ascontiguousarray(mask, dtype=np.uint8)).to(device)
    return DeviceSet(frames=frames, bias=masters[0], dark=masters[1], flat=masters[2],
                     exptime=np.ascontiguousarray(fs.exptime, dtype=np.float32),
                     dx=np.ascontiguousarray(fs.dx, dtype=np.float64),
                     dy=np.ascontiguousarray(fs.dy, dtype=np.float64),
                     mask=mask, saturation=float(saturation))


def _irp_sets(sets):
    arr = (IrpSet * len(sets))()
    keep = []
    dp = ctypes.POINTER(ctypes.c_double)
    fp = ctypes.POINTER(ctypes.c_float)
    for i, s in enumerate(sets):
        ptrs = (ctypes.c_void_p * s.n)(*[f.data_ptr() for f in s.frames])
        dx = np.ascontiguousarray(s.dx, dtype=np.float64)
        dy = np.ascontiguousarray(s.dy, dtype=np.float64)
        t = np.ascontiguousarray(s.exptime, dtype=np.float32)
        keep += [ptrs, dx, dy, t]
        a = arr[i]
        a.frames = ctypes.cast(ptrs, ctypes.POINTER(ctypes.c_void_p))
        a.raw_pitch = s.frames[0].stride(0)
        a.W, a.H, a.n = s.W, s.H, s.n
        a.dx = dx.ctypes.data_as(dp)
        a.dy = dy.ctypes.data_as(dp)
        a.exptime = t.ctypes.data_as(fp)
        a.bias, a.dark_rate, a.flat = s.bias.data_ptr(), s.dark.data_ptr(), s.flat.data_ptr()
        a.master_pitch = s.bias.stride(0)
        a.mean_out = s.mean.data_ptr() if s.mean is not None else None
        a.median_out = s.median.data_ptr() if s.median is not None else None
        a.nkept_out = s.nkept.data_ptr() if s.nkept is not None else None
        a.out_pitch = s.W
        a.stack_out = s.stack.data_ptr() if s.stack is not None else None
        a.ready_flag = s.ready_flag.data_ptr() if s.ready_flag is not None else None
        a.ready_value = int(s.ready_value)
        a.mask = s.mask.data_ptr() if s.mask is not None else None
        a.mask_pitch = s.mask.stride(0) if s.mask is not None else 0
        a.saturation = float(s.saturation)
    return arr, keep


def reduce_params(interp="bilinear", clip=None, normalize_flat=False, persistent=False,
                  max_ctas=0, wait_spin_limit=0, rows_per_warp=0,
                  frame_norm="none", spline_onchip=False) -> ReduceParams:
    """``frame_norm``: "none", "zero" or "scale" per-frame normalisation of the
    samples to the set's first frame before the combine.  ``spline_onchip``:
    unmasked cubic-spline sets on the row pass take the tile kernel (less DRAM
    traffic) instead of the column pass and vertical-tap reduction (faster)."""
    return ReduceParams(INTERP[interp], clip if clip is not None else clip_params(),
                        int(normalize_flat), int(persistent), int(max_ctas), int(wait_spin_limit),
                        int(rows_per_warp), FRAME_NORM[frame_norm], int(bool(spline_onchip)))


def workspace_size(sets, params: ReduceParams) -> int:
    arr, _ = _irp_sets(sets)
    n = lib().irp_workspace_size(arr, len(sets), ctypes.byref(params))
    if n == 0:
        raise ValueError("irp_workspace_size rejected the sets/params")
    return int(n)


def reduce_sets(sets, params: ReduceParams, ws=None, stream=None):
    """Fused reduction of one or more DeviceSets (outputs written into them)."""
    arr, keep = _irp_sets(sets)
    L = lib()
    need = L.irp_workspace_size(arr, len(sets), ctypes.byref(params))
    if need == 0:
        raise ValueError("irp_workspace_size rejected the sets/params")
    if ws is None or ws.numel() < need:
        ws = workspace(need, sets[0].frames[0].device)
    check(L.irp_reduce_set(arr, len(sets), ctypes.byref(params), _vp(ws), ws.numel(),
                           _stream(stream)), "irp_reduce_set")
    del keep
    return ws


def reduce_sets_host(sets, host_raw, host_out, params: ReduceParams, ws=None, stream=None):
    """irp_reduce_set_host: ``host_raw`` [i] is a host uint16 tensor [n, H, W]
    (pinned for overlap) copied into ``sets[i]``'s device frames, and
    ``host_out`` [i] a (mean, median) pair of host float32 [H, W] tensors (or
    None) that receive its results; each set is uploaded, reduced and
    downloaded in turn, the copies overlapping the neighbouring sets' work."""
    arr, keep = _irp_sets(sets)
    L = lib()
    need = max(L.irp_workspace_size(ctypes.byref(a), 1, ctypes.byref(params)) for a in arr)
    if need == 0:
        raise ValueError("irp_workspace_size rejected the sets/params")
    if ws is None or ws.numel() < need:
        ws = workspace(need, sets[0].frames[0].device)
    io = (IrpHostIo * len(sets))()
    for i, (h, out) in enumerate(zip(host_raw, host_out)):
        n, H, W = h.shape
        ptrs = (ctypes.c_void_p * n)(*[h[k].data_ptr() for k in range(n)])
        keep.append(ptrs)
        io[i].frames = ctypes.cast(ptrs, ctypes.POINTER(ctypes.c_void_p))
        io[i].pitch = h.stride(1)
        if out is not None:
            io[i].mean, io[i].median = out[0].data_ptr(), out[1].data_ptr()
            io[i].out_pitch = out[0].stride(0)
    check(L.irp_reduce_set_host(arr, len(sets), io, ctypes.byref(params), _vp(ws), ws.numel(),
                                _stream(stream)), "irp_reduce_set_host")
    del keep
    return ws


def sync_status(ws, stream=None) -> int:
    """Synchronises the stream and returns (and clears) the latched device status."""
    return int(lib().irp_sync_status(_vp(ws), _stream(stream)))


class Plan:
    """A reduction plan encoded into pinned host memory (CUDA-graph capturable).

    ``launch()`` issues one host->device copy of the plan and the kernels; a
    CUDA graph captured around ``launch()`` re-reads the pinned plan at each
    replay, so ``encode()`` may refresh offsets/pointers of the same shapes."""

    def __init__(self, sets, params: ReduceParams, device="cuda", ws=None):
        self.sets = list(sets)
        self.params = params
        arr, keep = _irp_sets(self.sets)
        L = lib()
        self.nbytes = int(L.irp_plan_bytes(arr, len(self.sets), ctypes.byref(params)))
        if self.nbytes == 0:
            raise ValueError("irp_plan_bytes rejected the sets/params")
        self.ws_bytes = int(L.irp_workspace_size(arr, len(self.sets), ctypes.byref(params)))
        self.host = torch.empty(self.nbytes, dtype=torch.uint8, pin_memory=True)
        self.ws = ws if (ws is not None and ws.numel() >= self.ws_bytes) else workspace(
            self.ws_bytes, device)
        self.encode()

    def encode(self, sets=None):
        if sets is not None:
            self.sets = list(sets)
        arr, keep = _irp_sets(self.sets)
        check(lib().irp_plan_encode(arr, len(self.sets), ctypes.byref(self.params),
                                    _vp(self.host), self.nbytes, _vp(self.ws), self.ws.numel()),
              "irp_plan_encode")

    def launch(self, stream=None):
        check(lib().irp_plan_launch(_vp(self.host), self.nbytes, _vp(self.ws), self.ws.numel(),
                                    _stream(stream)), "irp_plan_launch")


def profile_enable(on: bool = True) -> None:
    """Brackets every library launch with CUDA events (see irp_profile_read)."""
    lib().irp_profile_enable(int(bool(on)))


def profile_read() -> dict:
    """{kernel kind: (total ms, launches)} since the last read (synchronises)."""
    n = len(KERNEL_KINDS)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int64 * n)()
    k = lib().irp_profile_read(ctypes.cast(ms, ctypes.c_void_p), ctypes.cast(cnt, ctypes.c_void_p), n)
    return {KERNEL_KINDS[i]: (float(ms[i]), int(cnt[i])) for i in range(k)}

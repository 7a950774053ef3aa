"""FP64 CPU oracle of the image-reduction hot path (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Imported by the test suite, by the package smoke
check and by the benchmark's CPU-baseline leg; the product path never imports
it and shares no code with it.  The arithmetic lives in ``oracle.c`` (plain C,
double precision); this module only compiles and marshals.

Function pins (what checks the oracle against something other than itself)
are listed in ``tests/test_oracle.py``; ``tests/test_oracle_mutants.py``
compiles copies of ``oracle.c`` with planted mistakes (``compile_library``,
``load``) and checks that every one of them fails a pin.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

NEAREST, BILINEAR, SPLINE3, CUBIC = 0, 1, 2, 3
INTERP = {"nearest": NEAREST, "bilinear": BILINEAR, "spline3": SPLINE3, "cubic": CUBIC}
FRAME_NORM = {"none": 0, "zero": 1, "scale": 2}


class ClipParams(ctypes.Structure):
    _fields_ = [("kappa_lo", ctypes.c_double), ("kappa_hi", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("center", ctypes.c_int), ("ddof", ctypes.c_int)]


def clip_params(kappa=3.0, max_iter=3, center="mean", ddof=0, kappa_lo=None, kappa_hi=None):
    return ClipParams(float(kappa if kappa_lo is None else kappa_lo),
                      float(kappa if kappa_hi is None else kappa_hi), int(max_iter),
                      1 if center == "median" else 0, int(ddof))


def compile_library(src: str, out: str) -> str:
    """Compiles one oracle source file into a shared library at ``out`` with
    gcc (OpenMP when available).  The test suite also compiles deliberately
    broken copies of the source this way to check that its pins fail."""
    tmp = out + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-I" + _HERE, src, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:6] + ["-fopenmp"] + base[6:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compiles liboracle.so from oracle.c unless it is up to date."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        return _LIB
    return compile_library(_SRC, _LIB)


def load(path: str):
    """Loads an oracle shared library and declares its function signatures."""
    L = ctypes.CDLL(path)
    d, i, i64, p = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
    L.oracle_bspline3.restype = d
    L.oracle_bspline3.argtypes = [d]
    L.oracle_keys.restype = d
    L.oracle_keys.argtypes = [d]
    L.oracle_mirror.restype = i64
    L.oracle_mirror.argtypes = [i64, i64]
    L.oracle_mean_f32.restype = d
    L.oracle_mean_f32.argtypes = [p, i64, i, i]
    L.oracle_calibrate.restype = None
    L.oracle_calibrate.argtypes = [p, i64, i, i, p, p, p, i64, d, d, p]
    L.oracle_spline_solve_line.restype = None
    L.oracle_spline_solve_line.argtypes = [p, i64, p, i64, i, p]
    L.oracle_spline_coeffs.restype = None
    L.oracle_spline_coeffs.argtypes = [p, i, i, p]
    L.oracle_sample.restype = i
    L.oracle_sample.argtypes = [p, i, i, i, i, d, d, i, p]
    L.oracle_shift.restype = None
    L.oracle_shift.argtypes = [p, i, i, d, d, i, p, p]
    L.oracle_clip.restype = None
    L.oracle_clip.argtypes = [p, p, i, ctypes.POINTER(ClipParams), p, p, p, p, p]
    L.oracle_median.restype = d
    L.oracle_median.argtypes = [p, p, i]
    L.oracle_combine_stack.restype = None
    L.oracle_combine_stack.argtypes = [p, p, i, i64, ctypes.POINTER(ClipParams), i,
                                       p, p, p, p, p, p]
    L.oracle_reduce_set.restype = i
    L.oracle_reduce_set.argtypes = [p, i64, i64, i, i, i, p, p, p, i64, p, p, p, i, i,
                                    ctypes.POINTER(ClipParams), i, i64, p, p,
                                    p, p, p, p, p, p, p]
    L.oracle_reduce_set_masked.restype = i
    L.oracle_reduce_set_masked.argtypes = [p, i64, i64, i, i, i, p, p, p, i64, p, p, p,
                                           i, i, p, i64, d,
                                           ctypes.POINTER(ClipParams), i, i64, p, p,
                                           p, p, p, p, p, p, p, i]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load(build())
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def bspline3(t: float) -> float:
    return lib().oracle_bspline3(float(t))


def keys(t: float) -> float:
    """Keys' cubic convolution kernel, a = -1/2."""
    return lib().oracle_keys(float(t))


def mirror(i: int, N: int) -> int:
    return int(lib().oracle_mirror(int(i), int(N)))


def calibrate(raw, bias, dark, flat, t, normalize_flat=False):
    raw = np.ascontiguousarray(raw, dtype=np.uint16)
    bias = np.ascontiguousarray(bias, dtype=np.float32)
    dark = np.ascontiguousarray(dark, dtype=np.float32)
    flat = np.ascontiguousarray(flat, dtype=np.float32)
    H, W = raw.shape
    L = lib()
    norm = L.oracle_mean_f32(_ptr(flat), W, W, H) if normalize_flat else 1.0
    v = np.empty((H, W), dtype=np.float64)
    L.oracle_calibrate(_ptr(raw), W, W, H, _ptr(bias), _ptr(dark), _ptr(flat), W,
                       float(t), float(norm), _ptr(v))
    return v


def spline_solve_line(v):
    v = np.ascontiguousarray(v, dtype=np.float64)
    N = v.shape[0]
    c = np.empty(N, dtype=np.float64)
    work = np.empty(2 * N, dtype=np.float64)
    lib().oracle_spline_solve_line(_ptr(v), 1, _ptr(c), 1, N, _ptr(work))
    return c


def spline_coeffs(v):
    v = np.ascontiguousarray(v, dtype=np.float64)
    H, W = v.shape
    c = np.empty_like(v)
    lib().oracle_spline_coeffs(_ptr(v), W, H, _ptr(c))
    return c


def sample(f, x, y, dx, dy, interp):
    """One resampled value from frame data f (coefficients for spline3)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    H, W = f.shape
    out = np.zeros(1, dtype=np.float64)
    ok = lib().oracle_sample(_ptr(f), W, H, int(x), int(y), float(dx), float(dy),
                             INTERP.get(interp, interp), _ptr(out))
    return (float(out[0]) if ok else None)


def shift(v, dx, dy, interp):
    v = np.ascontiguousarray(v, dtype=np.float64)
    H, W = v.shape
    a = np.empty_like(v)
    valid = np.empty((H, W), dtype=np.uint8)
    lib().oracle_shift(_ptr(v), W, H, float(dx), float(dy), INTERP.get(interp, interp),
                       _ptr(a), _ptr(valid))
    return a, valid.astype(bool)


def clip(x, valid=None, adu=False, **kw):
    """(mean, kept, rejected, margin); with ``adu`` also the margin in the
    data's units (the smallest | |x - centre| - kappa sigma | of any pass)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    valid = np.ones(n, np.uint8) if valid is None else np.ascontiguousarray(valid, np.uint8)
    mean = np.zeros(1)
    kept = np.zeros(1, dtype=np.int32)
    rej = np.zeros(n, dtype=np.uint8)
    mg = np.zeros(1)
    mga = np.zeros(1)
    cp = clip_params(**kw)
    lib().oracle_clip(_ptr(x), _ptr(valid), n, ctypes.byref(cp), _ptr(mean), _ptr(kept),
                      _ptr(rej), _ptr(mg), _ptr(mga))
    out = (float(mean[0]), int(kept[0]), rej.astype(bool), float(mg[0]))
    return out + (float(mga[0]),) if adu else out


def median(x, valid=None):
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    valid = np.ones(n, np.uint8) if valid is None else np.ascontiguousarray(valid, np.uint8)
    return float(lib().oracle_median(_ptr(x), _ptr(valid), n))


def combine_stack(stack, valid, nthreads=1, **kw):
    """Per-pixel clip + median over an aligned stack [n, H, W] (FP64 in, FP64 out)."""
    stack = np.ascontiguousarray(stack, dtype=np.float64)
    n = stack.shape[0]
    shape = stack.shape[1:]
    P = int(np.prod(shape))
    valid = np.ascontiguousarray(valid, dtype=np.uint8)
    mean = np.empty(shape)
    med = np.empty(shape)
    kept = np.empty(shape, dtype=np.int32)
    margin = np.empty(shape)
    margin_adu = np.empty(shape)
    rej = np.empty(stack.shape, dtype=np.uint8)
    cp = clip_params(**kw)
    lib().oracle_combine_stack(_ptr(stack), _ptr(valid), n, P, ctypes.byref(cp), int(nthreads),
                               _ptr(mean), _ptr(med), _ptr(kept), _ptr(margin),
                               _ptr(margin_adu), _ptr(rej))
    return dict(mean=mean, median=med, nkept=kept, margin=margin, margin_adu=margin_adu,
                rejected=rej.astype(bool))


def reduce_set(fs, interp="bilinear", kappa=3.0, max_iter=3, center="mean", ddof=0,
               normalize_flat=False, nthreads=1, pixels=None, want_stack=False,
               kappa_lo=None, kappa_hi=None, mask=None, saturation=None, frame_norm="none"):
    """Whole frame set -> dict(mean, median, nkept, margin, margin_adu[, stack, valid]).

    ``mask`` ([H,W] uint8, non-zero = bad) and ``saturation`` (raw ADU) mark
    bad source pixels (Sec. 2.1 bad-pixel masking): a sample whose taps with
    non-zero weight include a bad pixel is invalid.

    ``fs`` is a ``synth.FrameSet``-like object (raw [n,H,W] u16, masters [H,W]
    f32, exptime [n], dx/dy [n]).  ``pixels`` = (xs, ys) restricts the output
    to those pixels (returned as 1-D arrays).  ``frame_norm`` ("none", "zero",
    "scale") normalises each frame's samples to frame 0 by the frames' mean
    calibrated levels before the combine."""
    raw = np.ascontiguousarray(fs.raw, dtype=np.uint16)
    n, H, W = raw.shape
    bias = np.ascontiguousarray(fs.bias, np.float32)
    dark = np.ascontiguousarray(fs.dark, np.float32)
    flat = np.ascontiguousarray(fs.flat, np.float32)
    t = np.ascontiguousarray(fs.exptime, np.float64)
    dx = np.ascontiguousarray(fs.dx, np.float64)
    dy = np.ascontiguousarray(fs.dy, np.float64)
    cp = clip_params(kappa, max_iter, center, ddof, kappa_lo, kappa_hi)
    if pixels is not None:
        px = np.ascontiguousarray(pixels[0], np.int32)
        py = np.ascontiguousarray(pixels[1], np.int32)
        npix = px.shape[0]
        shape = (npix,)
    else:
        px = py = np.zeros(1, np.int32)
        npix = 0
        shape = (H, W)
    mean = np.empty(shape)
    med = np.empty(shape)
    kept = np.empty(shape, np.int32)
    margin = np.empty(shape)
    margin_adu = np.empty(shape)
    stack = np.empty((n, H, W)) if (want_stack and pixels is None) else None
    valid = np.empty((n, H, W), np.uint8) if (want_stack and pixels is None) else None
    mk = np.ascontiguousarray(mask, np.uint8) if mask is not None else None
    rc = lib().oracle_reduce_set_masked(
        _ptr(raw), W, H * W, W, H, n, _ptr(bias), _ptr(dark), _ptr(flat), W, _ptr(t),
        _ptr(dx), _ptr(dy), INTERP.get(interp, interp), int(bool(normalize_flat)),
        _ptr(mk) if mk is not None else None, W,
        float(saturation) if saturation is not None else 0.0,
        ctypes.byref(cp), int(nthreads), int(npix), _ptr(px), _ptr(py),
        _ptr(mean), _ptr(med), _ptr(kept), _ptr(margin), _ptr(margin_adu),
        _ptr(stack) if stack is not None else None,
        _ptr(valid) if valid is not None else None,
        FRAME_NORM[frame_norm])
    if rc == 2:
        raise ValueError("oracle_reduce_set: a frame's mean is 0 or not finite (scale)")
    if rc != 0:
        raise ValueError("oracle_reduce_set rejected its arguments")
    out = dict(mean=mean, median=med, nkept=kept, margin=margin, margin_adu=margin_adu)
    if stack is not None:
        out["stack"] = stack
        out["valid"] = valid.astype(bool)
    return out


def relative_difference(img, ref):
    """Delta I_ij = (I_ij - I_ref_ij) / I_ref_ij (Sec. 3.1, the relative-difference
    image used for every consistency check in the paper)."""
    img = np.asarray(img, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return (img - ref) / ref


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))

"""Shared helpers of the GPU parity tests: uploads, oracle runs and the
tolerances derived from the FP32 arithmetic of the kernels.

Tolerances, each derived from the rounding steps of the FP32 arithmetic.
Calibration is v = (raw - L) * rf with the level L = bias + dark*t rounded
once (an fma) and rf = flat_norm/flat: its error is at most
u (|L| rf + 3 |v|), so below "|v|" stands for |v| + |L| rf.
  * clipped mean / median end to end:  |gpu - ref| <= max(1e-3 ADU, 1e-6 |ref|)
    plus the per-sample bound below (the mean of samples is off by at most
    the largest sample error);
  * one resampled sample, nearest / bilinear: 8 u M3 + 1e-5, M3 = largest
    |v| among the 3x3 source pixels around the tap origin (calibration and
    two lerps, each a few roundings of values bounded by M3), u = 2^-24;
  * one resampled sample, Keys cubic convolution: 16 u M5 + 1e-5, M5 = largest
    |v| in the 5x5 neighbourhood (calibration, then two 4-tap passes whose
    weights have an absolute sum of at most 1.25 per axis);
  * one resampled sample, cubic spline: 64 u M9 + 1e-4, M9 = largest |v|
    within 4 px of the tap origin (recursive prefilter of gain sqrt(3) per
    direction and axis; error terms of farther pixels decay as 0.268^d);
  * median on identical inputs: bit-exact; clip masks on identical inputs:
    identical except at pixels the oracle marks within 1e-5 sigma of a
    threshold.

End to end (GPU from raw against the FP64 oracle from raw), ``gate_e2e``:
  * clip results (kept counts) must agree, except where the oracle's smallest
    threshold distance in ADU is within (2 + kappa) times the pixel's sample
    bound: a sample error e moves |x - mu| by at most 2|e| and kappa sigma by
    at most kappa |e|, so no larger distance can flip a decision;
  * the mean and median within max(1e-3 ADU, 1e-6 |ref|) (the target
    bound of the path, read as atol + rtol) at every compared pixel where the sample
    rounding bound (a-priori, or the measured sample errors when the stack
    is at hand) stays inside it; elsewhere -- next to bright stars, where the
    spline's FP32 prefilter carries rounding from coefficients far larger
    than the pixel -- within it plus that bound, on at most 1e-3 of the
    pixels.  The fraction of pixels outside the plain tolerance is reported.
"""
import numpy as np

U = 2.0 ** -24


def maxfilter(a, size):
    from scipy.ndimage import maximum_filter
    return maximum_filter(np.abs(a), size=size, mode="nearest")


def sample_tolerance(fs, interp, oracle_mod, pixels=None):
    """Per-sample tolerance [n,H,W] of the aligned stack on the output grid,
    or [n, len(xs)] at the output pixels ``pixels`` = (xs, ys)."""
    n, H, W = fs.raw.shape
    size, coef, floor_ = {"spline3": (9, 64.0, 1e-4), "cubic": (5, 16.0, 1e-5)}.get(
        interp, (3, 8.0, 1e-5))
    if pixels is not None:
        return _sample_tolerance_at(fs, oracle_mod, pixels, size, coef, floor_)
    yy, xx = np.mgrid[0:H, 0:W]
    tol = np.empty((n,) + xx.shape)
    for k in range(n):
        v = oracle_mod.calibrate(fs.raw[k], fs.bias, fs.dark, fs.flat, fs.exptime[k])
        lv = np.abs(fs.bias.astype(np.float64) + fs.dark.astype(np.float64) * float(fs.exptime[k]))
        M = maxfilter(np.abs(v) + lv / np.abs(fs.flat.astype(np.float64)), size)
        sx = np.clip(xx + int(np.floor(fs.dx[k])), 0, W - 1)
        sy = np.clip(yy + int(np.floor(fs.dy[k])), 0, H - 1)
        # the tap origin and its right/upper neighbour
        sx1 = np.clip(sx + 1, 0, W - 1)
        sy1 = np.clip(sy + 1, 0, H - 1)
        m = np.maximum(np.maximum(M[sy, sx], M[sy, sx1]), np.maximum(M[sy1, sx], M[sy1, sx1]))
        tol[k] = coef * U * m + floor_
    return tol


def _sample_tolerance_at(fs, oracle_mod, pixels, size, coef, floor_):
    """sample_tolerance at the given output pixels only: the same maxima,
    taken over each pixel's own window of calibrated values (the size x size
    maxima at the tap origin and its right/upper neighbour cover rows and
    columns origin - h .. origin + h + 1, clamped to the frame as the
    full-frame filter's nearest mode clamps them), so that a full-size set
    needs no pass over whole frames."""
    n, H, W = fs.raw.shape
    xx, yy = (np.asarray(a) for a in pixels)
    h = size // 2
    offs = np.arange(-h, h + 2)
    K = offs.size
    tol = np.empty((n,) + xx.shape)
    for k in range(n):
        sx = np.clip(xx + int(np.floor(fs.dx[k])), 0, W - 1).reshape(-1)
        sy = np.clip(yy + int(np.floor(fs.dy[k])), 0, H - 1).reshape(-1)
        Y = np.clip(sy[:, None] + offs[None, :], 0, H - 1)[:, :, None]
        X = np.clip(sx[:, None] + offs[None, :], 0, W - 1)[:, None, :]
        shape2 = (sx.size, K * K)
        raw = np.ascontiguousarray(fs.raw[k][Y, X].reshape(shape2))
        bias = fs.bias[Y, X].reshape(shape2)
        dark = fs.dark[Y, X].reshape(shape2)
        flat = fs.flat[Y, X].reshape(shape2)
        v = oracle_mod.calibrate(raw, bias, dark, flat, fs.exptime[k])
        lv = np.abs(bias.astype(np.float64) + dark.astype(np.float64) * float(fs.exptime[k]))
        m = (np.abs(v) + lv / np.abs(flat.astype(np.float64))).max(axis=1)
        tol[k] = (coef * U * m + floor_).reshape(xx.shape)
    return tol


def mean_tolerance(ref):
    return np.maximum(1e-3, 1e-6 * np.abs(ref))


def compare(name, got, ref, tol, mask=None):
    """Asserts |got - ref| <= tol where mask (and both finite); returns stats."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    both_nan = np.isnan(got) & np.isnan(ref)
    m = ~both_nan if mask is None else (mask & ~both_nan)
    assert not np.any(np.isnan(got[m]) != np.isnan(ref[m])), f"{name}: NaN pattern differs"
    fin = m & np.isfinite(ref)
    err = np.abs(got - ref)
    bad = fin & (err > tol)
    ratio = np.max(err[fin] / np.broadcast_to(tol, err.shape)[fin]) if fin.any() else 0.0
    assert not bad.any(), (f"{name}: {bad.sum()} of {fin.sum()} outside tolerance, "
                           f"worst err {err[bad].max():.3g} at ratio {ratio:.3g}")
    return dict(max_err=float(err[fin].max()) if fin.any() else 0.0, max_ratio=float(ratio))


def gate_e2e(name, got, ref, samp, kappa, meas=None, max_outside=1e-3):
    """End-to-end gate of one set's outputs (see the module docstring).

    got: dict with mean, median, nkept (arrays over the compared pixels);
    ref: the oracle's reduce_set dict (mean, median, nkept, margin, margin_adu);
    samp: per-pixel a-priori sample bound (max over the pixel's frames);
    meas: per-pixel measured largest sample error |gpu - oracle| (optional;
    when given it replaces the a-priori bound in the mean/median gates);
    max_outside: cap on the fraction of compared pixels outside the plain
    tolerance (None: no cap).  Returns the statistics."""
    gm = np.asarray(got["mean"], np.float64)
    gd = np.asarray(got["median"], np.float64)
    samp = np.broadcast_to(np.asarray(samp, np.float64), gm.shape)
    allowed = (ref["margin_adu"] < (2.0 + kappa) * samp) | (ref["margin"] < 1e-5)
    if got.get("nkept") is None:
        # no kept counts to compare: the mean is gated where no decision can flip
        mismatch = allowed
    else:
        gk = np.asarray(got["nkept"]).astype(np.int64)
        rk = np.asarray(ref["nkept"]).astype(np.int64)
        mismatch = gk != rk
        bad = mismatch & ~allowed
        assert not bad.any(), (f"{name}: clip results differ at {int(bad.sum())} pixels whose "
                               f"threshold distance exceeds the rounding reach")
    extra = samp if meas is None else np.broadcast_to(np.asarray(meas, np.float64), gm.shape)
    stats = {"pixels": int(gm.size), "clip_mismatch_frac": float(mismatch.mean())}
    for key, g in (("mean", gm), ("median", gd)):
        r = np.asarray(ref[key], np.float64)
        cmp = ~mismatch if key == "mean" else np.ones(gm.shape, bool)
        plain = mean_tolerance(r)
        compare(f"{name} {key}", g, r, plain + extra, cmp)
        attain = extra <= plain
        compare(f"{name} {key} (plain tolerance)", g, r, plain, cmp & attain)
        fin = cmp & np.isfinite(r)
        err = np.abs(g - r)
        outside = fin & (err > plain)
        stats[f"{key}_max_abs"] = float(err[fin].max()) if fin.any() else 0.0
        stats[f"{key}_max_rel"] = float((err[fin] / np.maximum(np.abs(r[fin]), 1e-30)).max()) \
            if fin.any() else 0.0
        stats[f"{key}_outside_plain_frac"] = float(outside.sum() / max(fin.sum(), 1))
        stats[f"{key}_bound_above_plain_frac"] = float((fin & ~attain).sum() / max(fin.sum(), 1))
        if max_outside is not None:
            assert stats[f"{key}_outside_plain_frac"] <= max_outside, (name, key, stats)
    return stats

"""Pins of the FP64 oracle against values fixed by the paper and by mathematics.

Each check compares the oracle with something other than itself: hand-worked
values (tests/golden), closed forms (the cubic B-spline basis image of
Sec. 3.1.1, bilinear polynomials, Samuelson's bound), a dense solve of the
spline system built from the basis function and the boundary rule, and numpy's
median.  None of these tests needs a GPU.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2008_11486_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line)
    return rows


# ---------------------------------------------------------------- B-spline basis
def test_bspline3_golden_values():
    for row in _read_golden("bspline3_values.txt"):
        t, num, den = row.split()
        assert oracle.bspline3(float(t)) == pytest.approx(int(num) / int(den), abs=1e-15)


def test_bspline3_partition_of_unity_and_moments():
    # sum_k beta3(t - k) = 1 and sum_k k beta3(t - k) = t for every t
    for t in np.linspace(-3.0, 3.0, 61):
        w = [oracle.bspline3(t - k) for k in range(-6, 7)]
        assert sum(w) == pytest.approx(1.0, abs=1e-14)
        assert sum(k * wk for k, wk in zip(range(-6, 7), w)) == pytest.approx(t, abs=1e-13)


def test_keys_golden_values():
    for row in _read_golden("keys_values.txt"):
        t, num, den = row.split()
        assert oracle.keys(float(t)) == pytest.approx(int(num) / int(den), abs=1e-15)


def test_keys_reproduces_quadratics():
    # a = -1/2 makes cubic convolution exact on polynomials up to degree 2:
    # sum_k W(t - k) k^m = t^m for m = 0, 1, 2
    for t in np.linspace(-3.0, 3.0, 61):
        w = [oracle.keys(t - k) for k in range(-6, 7)]
        for m in range(3):
            assert sum(wk * k ** m for k, wk in zip(range(-6, 7), w)) == \
                pytest.approx(t ** m, abs=1e-12)


def test_keys_shift_of_a_quadratic_image_is_exact():
    """Cubic convolution shifts a quadratic surface exactly wherever all its
    taps lie inside the frame; integer offsets are pure pixel moves."""
    H, W = 20, 24
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    surf = lambda X, Y: 3.0 + 0.5 * X - 0.25 * Y + 0.01 * X * X + 0.02 * X * Y - 0.03 * Y * Y
    v = surf(xx, yy)
    for dx, dy in [(0.3, -1.7), (2.25, 0.5), (-0.75, 3.1)]:
        a, ok = oracle.shift(v, dx, dy, "cubic")
        want = surf(xx + dx, yy + dy)
        assert ok.sum() > 0
        np.testing.assert_allclose(a[ok], want[ok], atol=1e-11)
        # valid iff the 4 taps of each axis lie inside: i0 - 1 >= 0 and i0 + 2 <= N - 1
        i0 = xx + np.floor(dx)
        j0 = yy + np.floor(dy)
        want_ok = (i0 >= 1) & (i0 <= W - 3) & (j0 >= 1) & (j0 <= H - 3)
        assert np.array_equal(ok, want_ok)
    # an integer shift reads only the tap it lands on: a pixel move, valid up
    # to the frame edge
    a, ok = oracle.shift(v, 2.0, -3.0, "cubic")
    assert ok[3:, : W - 2].all() and not ok[:3].any() and not ok[:, W - 2:].any()
    assert np.array_equal(a[3:, : W - 2], v[: H - 3, 2:])


def test_mirror_index():
    assert [oracle.mirror(i, 5) for i in range(-4, 13)] == \
        [4, 3, 2, 1, 0, 1, 2, 3, 4, 3, 2, 1, 0, 1, 2, 3, 4]
    assert oracle.mirror(-7, 1) == 0 and oracle.mirror(5, 1) == 0
    assert [oracle.mirror(i, 2) for i in range(-3, 4)] == [1, 0, 1, 0, 1, 0, 1]


# ---------------------------------------------------------------- calibration
def test_calibrate_golden_3x3():
    rows = {r.split()[0]: r.split()[1:] for r in _read_golden("calibrate_3x3.txt")}
    t = float(rows["t"][0])
    raw = np.array(rows["raw"], dtype=np.float64).astype(np.uint16).reshape(3, 3)
    bias = np.array(rows["bias"], dtype=np.float32).reshape(3, 3)
    dark = np.array(rows["dark"], dtype=np.float32).reshape(3, 3)
    flat = np.array(rows["flat"], dtype=np.float32).reshape(3, 3)
    want = np.array(rows["v"], dtype=np.float64).reshape(3, 3)
    got = oracle.calibrate(raw, bias, dark, flat, t)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-5)


def test_calibrate_constant_closed_form_and_flat_normalisation():
    raw = np.full((4, 6), 1234, np.uint16)
    v = oracle.calibrate(raw, np.full((4, 6), 1000.5, np.float32), np.full((4, 6), 0.0625, np.float32),
                         np.full((4, 6), 0.8, np.float32), 60.0)
    # (1234 - 1000.5 - 3.75) / 0.8 = 229.75 / 0.8
    np.testing.assert_allclose(v, 229.75 / np.float64(np.float32(0.8)), rtol=1e-15)
    # normalised flat: flat' = flat / mean(flat); flat = [1, 3] -> mean 2 -> [0.5, 1.5]
    flat = np.tile(np.array([1.0, 3.0], np.float32), (2, 1))
    raw2 = np.full((2, 2), 1100, np.uint16)
    v2 = oracle.calibrate(raw2, np.full((2, 2), 1000, np.float32), np.zeros((2, 2), np.float32),
                          flat, 60.0, normalize_flat=True)
    np.testing.assert_allclose(v2, [[200.0, 100.0 / 1.5]] * 2, rtol=1e-15)


# ---------------------------------------------------------------- spline system
def _dense_mirror_system(N):
    """Matrix of the interpolation condition sum_i c_ext[i] beta3(j - i) = v[j],
    c_ext the mirror extension of c, assembled from beta3 and the index map."""
    A = np.zeros((N, N))
    for j in range(N):
        for i in range(j - 2, j + 3):
            A[j, oracle.mirror(i, N)] += oracle.bspline3(j - i)
    return A


@pytest.mark.parametrize("N", [1, 2, 3, 5, 17, 64])
def test_spline_line_solve_equals_dense_system(N):
    rng = np.random.default_rng(N)
    v = rng.normal(size=N) * 100
    c = oracle.spline_solve_line(v)
    A = _dense_mirror_system(N)
    np.testing.assert_allclose(c, np.linalg.solve(A, v), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(A @ c, v, rtol=1e-12, atol=1e-11)


def test_spline_line_reproduces_basis_and_mirror_pair():
    N = 20
    # a basis function at an interior knot: coefficients are a unit impulse
    v = np.array([oracle.bspline3(j - 9) for j in range(N)])
    c = oracle.spline_solve_line(v)
    want = np.zeros(N)
    want[9] = 1.0
    np.testing.assert_allclose(c, want, atol=1e-14)
    # data symmetric about sample 0 (beta3(j-1)+beta3(j+1)) is consistent with the
    # mirror boundary: its coefficients are the impulse at 1 alone
    v = np.array([oracle.bspline3(j - 1) + oracle.bspline3(j + 1) for j in range(N)])
    c = oracle.spline_solve_line(v)
    want = np.zeros(N)
    want[1] = 1.0
    np.testing.assert_allclose(c, want, atol=1e-14)
    # the same at the right end
    v = np.array([oracle.bspline3(j - (N - 2)) + oracle.bspline3(j - N) for j in range(N)])
    c = oracle.spline_solve_line(v)
    want = np.zeros(N)
    want[N - 2] = 1.0
    np.testing.assert_allclose(c, want, atol=1e-14)


def _bspline_basis_image(W, H, centres, amps, dx=0.0, dy=0.0):
    """Sum of 2-D cubic B-spline basis functions sampled at (x+dx, y+dy)."""
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    img = np.zeros((H, W))
    b = np.vectorize(oracle.bspline3)
    for (cx, cy), a in zip(centres, amps):
        img += a * b(xx + dx - cx) * b(yy + dy - cy)
    return img


def test_spline3_shift_exact_on_bspline_basis_image():
    """Sec. 3.1.1: an image of cubic B-spline basis functions can be shifted
    without interpolating; the spline shift must reproduce it (the paper's own
    accuracy test).  Centres on the frame edge are mirror-consistent too."""
    W, H = 40, 33
    rng = np.random.default_rng(5)
    centres = [(int(rng.integers(2, W - 2)), int(rng.integers(2, H - 2))) for _ in range(25)]
    centres += [(0, 10), (W - 1, 20), (15, 0), (30, H - 1), (0, 0)]
    amps = rng.uniform(100, 5000, size=len(centres))
    img = _bspline_basis_image(W, H, centres, amps) + 300.0 * 0  # no offset term
    for dx, dy in [(0.3, 0.2), (0.6, 0.7), (-1.75, 2.5), (3.0, -2.0), (0.0, 0.0)]:
        a, valid = oracle.shift(img, dx, dy, "spline3")
        want = _bspline_basis_image(W, H, centres, amps, dx, dy)
        err = np.abs(a - want)[valid]
        assert valid.sum() > 0.7 * W * H
        assert err.max() <= 1e-11 * np.abs(img).max()


def test_spline3_interpolates_at_integer_shift():
    rng = np.random.default_rng(1)
    v = rng.normal(300, 20, size=(21, 19))
    a, valid = oracle.shift(v, 2.0, -3.0, "spline3")
    np.testing.assert_allclose(a[valid], np.roll(np.roll(v, -2, 1), 3, 0)[valid], atol=1e-10)
    assert valid[3:, :17].all() and not valid[:3].any() and not valid[:, 17:].any()


def test_spline3_round_trip_magnitude_like_paper():
    """Sec. 3.1.1 set B: shift by (0.6, 0.7) and back; the paper finds relative
    differences of about 1e-2 to 1e-1 on sky-dominated frames."""
    fs = synth.make_set(96, 96, 1, 0.0, 77)
    v = oracle.calibrate(fs.raw[0], fs.bias, fs.dark, fs.flat, 60.0)
    a, va = oracle.shift(v, 0.6, 0.7, "spline3")
    b, vb = oracle.shift(a, -0.6, -0.7, "spline3")
    d = np.abs(oracle.relative_difference(b, v))[20:-20, 20:-20]
    q90 = np.quantile(d, 0.9)
    assert 1e-3 < q90 < 2e-1


# ---------------------------------------------------------------- nearest / bilinear
@pytest.mark.parametrize("interp", ["nearest", "bilinear", "spline3"])
def test_zero_shift_is_identity(interp):
    rng = np.random.default_rng(3)
    v = rng.normal(300, 50, size=(13, 17))
    a, valid = oracle.shift(v, 0.0, 0.0, interp)
    assert valid.all()
    if interp == "spline3":
        np.testing.assert_allclose(a, v, atol=1e-10)
    else:
        assert np.array_equal(a, v)


@pytest.mark.parametrize("interp", ["nearest", "bilinear"])
def test_integer_shift_moves_pixels_exactly(interp):
    rng = np.random.default_rng(4)
    v = rng.normal(300, 50, size=(12, 15))
    a, valid = oracle.shift(v, -3.0, 2.0, interp)
    # output (x, y) = v(x - 3, y + 2): valid for x >= 3, y <= H - 3
    assert np.array_equal(valid[:, 3:][:-2], np.ones((10, 12), bool))
    assert not valid[:, :3].any() and not valid[-2:].any()
    assert np.array_equal(a[:-2, 3:], v[2:, :-3])


def test_bilinear_reproduces_bilinear_polynomials():
    """f = a + b x + c y + d x y is reproduced exactly by bilinear weights; a
    swapped or transposed weight breaks this."""
    H, W = 14, 11
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    f = lambda x, y: 3.0 + 0.7 * x - 1.3 * y + 0.11 * x * y
    v = f(xx, yy)
    for dx, dy in [(0.25, 0.5), (-2.375, 1.625), (0.9, -0.1)]:
        a, valid = oracle.shift(v, dx, dy, "bilinear")
        np.testing.assert_allclose(a[valid], f(xx + dx, yy + dy)[valid], rtol=1e-13, atol=1e-12)


def test_bilinear_midpoint_and_validity_edges():
    H, W = 6, 9
    ramp = np.tile(np.arange(W, dtype=np.float64) * 10, (H, 1))
    a, valid = oracle.shift(ramp, 0.5, 0.0, "bilinear")
    assert np.array_equal(a[:, :W - 1], ramp[:, :W - 1] + 5.0)
    assert valid[:, :W - 1].all() and not valid[:, W - 1].any()
    # dx = 1.5: i0 = x + 1, needs i0 + 1 <= W - 1 -> x <= W - 3
    # dy = -2.25: floor = -3, fy = 0.75, j0 = y - 3 >= 0 and j0 + 1 = y - 2 <= H - 1 -> y >= 3
    _, valid = oracle.shift(ramp, 1.5, -2.25, "bilinear")
    want = np.zeros((H, W), bool)
    want[3:H, 0:W - 2] = True
    assert np.array_equal(valid, want)


def test_nearest_rounds_half_away_from_zero():
    W = 6
    v = np.tile(np.arange(W, dtype=np.float64), (1, 1))
    # dx = 0.5: position x + 0.5 rounds up -> x + 1
    a, valid = oracle.shift(v, 0.5, 0.0, "nearest")
    assert np.array_equal(a[0, :W - 1], np.arange(1, W)) and not valid[0, W - 1]
    # dx = -0.5: position x - 0.5; x = 0 gives -0.5 -> -1 (invalid), x >= 1 -> x
    a, valid = oracle.shift(v, -0.5, 0.0, "nearest")
    assert not valid[0, 0] and np.array_equal(a[0, 1:], np.arange(1, W))
    # dx = 0.49 -> x, dx = 0.51 -> x + 1
    a, _ = oracle.shift(v, 0.49, 0.0, "nearest")
    assert np.array_equal(a[0], np.arange(W))
    a, valid = oracle.shift(v, 0.51, 0.0, "nearest")
    assert np.array_equal(a[0, :W - 1], np.arange(1, W)) and not valid[0, W - 1]


# ---------------------------------------------------------------- sigma clip / median
def test_clip_golden_cases():
    for row in _read_golden("clip_cases.txt"):
        name, params, samples, expect = [s.strip() for s in row.split("|")]
        klo, khi, it, center, ddof = params.split()
        x = np.array(samples.split(), dtype=np.float64)
        mean_want, kept_want = expect.split()
        mean, kept, rej, _ = oracle.clip(x, kappa_lo=float(klo), kappa_hi=float(khi),
                                         max_iter=int(it), center="median" if center == "1" else "mean",
                                         ddof=int(ddof))
        assert kept == int(kept_want), name
        assert mean == pytest.approx(float(mean_want), abs=1e-12), name
        assert rej.sum() == len(x) - kept, name


@pytest.mark.parametrize("m", [1, 2, 3, 5, 9, 10])
def test_clip_cannot_reject_at_kappa3_for_ten_or_fewer(m):
    """Samuelson: |x - mu| <= sigma sqrt(m - 1) <= 3 sigma for m <= 10, so the
    clipped mean is the plain mean."""
    rng = np.random.default_rng(m)
    for _ in range(50):
        x = rng.standard_cauchy(size=m) * 100
        mean, kept, _, _ = oracle.clip(x)
        assert kept == m
        assert mean == pytest.approx(np.mean(x), rel=1e-12, abs=1e-9)


def test_clip_without_outliers_is_plain_mean():
    x = np.linspace(-1.0, 1.0, 31) * 7 + 300
    mean, kept, _, _ = oracle.clip(x)
    assert kept == 31 and mean == pytest.approx(np.mean(x), rel=1e-15)


def test_clip_invalid_samples_are_excluded():
    x = np.array([1.0, 2.0, 1e9, 3.0])
    mean, kept, _, _ = oracle.clip(x, valid=np.array([1, 1, 0, 1]))
    assert kept == 3 and mean == pytest.approx(2.0)
    mean, kept, _, _ = oracle.clip(x, valid=np.zeros(4))
    assert kept == 0 and np.isnan(mean)
    assert np.isnan(oracle.median(x, valid=np.zeros(4)))


def test_clip_margin_reports_distance_to_threshold():
    # case B of the golden file sits exactly on the threshold
    _, _, _, mg = oracle.clip(np.array([0.0] * 9 + [10.0]))
    assert mg == 0.0
    _, _, _, mg = oracle.clip(np.array([5.0, 5.0]))
    assert mg == np.inf
    # 0 0 0 0 10 at kappa 3: mean 2, sigma^2 = (4*4 + 64)/5 = 16, threshold 12;
    # the 10 lies 8 from the mean, one sigma inside it (the zeros 2.5 sigma)
    _, kept, _, mg = oracle.clip(np.array([0.0, 0.0, 0.0, 0.0, 10.0]))
    assert kept == 5 and mg == pytest.approx(1.0, abs=1e-15)


def test_clip_margin_in_data_units_worked_by_hand():
    """The threshold distance in the data's units, | |x - centre| - kappa sigma |,
    the smallest over every sample of every pass (cases of the golden file)."""
    # A: 1..5, kappa 3: sigma = sqrt(2); the outer samples sit 3 sqrt(2) - 2 inside
    *_, mga = oracle.clip(np.arange(1.0, 6.0), adu=True)
    assert mga == pytest.approx(3 * np.sqrt(2) - 2, abs=1e-13)
    # C: ten 0 and one 11: pass 1 has mu 1, sigma sqrt(10); the 11 lies
    # 10 - 3 sqrt(10) beyond the threshold; pass 2 has sigma 0 and tests nothing
    *_, mg, mga = oracle.clip(np.array([0.0] * 10 + [11.0]), adu=True)
    assert mga == pytest.approx(10 - 3 * np.sqrt(10), abs=1e-13)
    assert mga == pytest.approx(mg * np.sqrt(10), abs=1e-13)
    # D: eight 0, 3, 100 at kappa 2.  Pass 1: mu 10.3, 2 sigma = 59.83, the
    # closest sample (100, |d| = 89.7) is 29.87 away.  Pass 2: eight 0 and 3,
    # mu 1/3, sigma sqrt(8)/3: the 3 lies 8/3 - 2 sqrt(8)/3 beyond 2 sigma, the
    # smallest distance of all (a zero lies 2 sqrt(8)/3 - 1/3 inside).
    x = np.array([0.0] * 8 + [3.0, 100.0])
    *_, mga = oracle.clip(x, adu=True, kappa=2.0)
    assert mga == pytest.approx(8 / 3 - 2 * np.sqrt(8) / 3, abs=1e-13)
    # asymmetric thresholds: F, nine 0 and 10 with kappa_hi 2: mu 1, sigma 3,
    # the 10 is 9 - 6 = 3 beyond, the zeros 9 - 1 = 8 inside kappa_lo 3
    *_, mga = oracle.clip(np.array([0.0] * 9 + [10.0]), adu=True, kappa_lo=3.0, kappa_hi=2.0)
    assert mga == pytest.approx(3.0, abs=1e-13)
    # G, the mirror image: nine 0 and -10 with kappa_lo 2: the -10 lies 9 below
    # the mean, 3 beyond 2 sigma (the zeros lie 8 inside kappa_hi 3)
    *_, mga = oracle.clip(np.array([0.0] * 9 + [-10.0]), adu=True, kappa_lo=2.0, kappa_hi=3.0)
    assert mga == pytest.approx(3.0, abs=1e-13)


def test_clip_result_is_a_fixed_point_of_the_rule():
    """Properties any correct run of the iteration has, checked on random small
    stacks with outliers (mean centre, ddof 0, passes until nothing changes):
    the survivors S reject nothing more (|x - mean(S)| <= kappa sigma(S), or
    sigma(S) = 0); every rejected sample lies outside [min S, max S], since
    each pass cuts both tails of the current survivors; the output is mean(S)
    and the count |S|."""
    rng = np.random.default_rng(20081)
    for trial in range(400):
        n = int(rng.integers(1, 9))
        x = rng.normal(0.0, 1.0, n)
        x[rng.random(n) < 0.25] += rng.choice([-1, 1]) * rng.uniform(3, 30)
        kappa = float(rng.choice([1.0, 1.5, 2.0, 2.5]))
        mean, kept, rej, _ = oracle.clip(x, kappa=kappa, max_iter=100)
        S = x[~rej]
        assert kept == S.size >= 1
        mu, sd = S.mean(), S.std()
        if sd > 0:
            assert np.all(np.abs(S - mu) <= kappa * sd * (1 + 1e-12)), (trial, x, kappa)
        assert np.all((x[rej] < S.min()) | (x[rej] > S.max())), (trial, x, kappa)
        assert mean == pytest.approx(mu, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 7, 10, 31, 40])
def test_median_matches_numpy(m):
    rng = np.random.default_rng(100 + m)
    for _ in range(20):
        x = rng.normal(size=m).astype(np.float32).astype(np.float64)
        valid = rng.random(m) < 0.8
        if not valid.any():
            continue
        assert oracle.median(x, valid) == np.median(x[valid])


# ---------------------------------------------------------------- whole set
@pytest.mark.parametrize("interp", ["nearest", "bilinear", "spline3"])
def test_reduce_set_constant_frames(interp):
    fs = synth.make_const_set(24, 20, 6, 1500, 1000.0, 0.05, 0.8, 60.0,
                              dx=[0.3, -1.7, 2.25, 0.0, -0.5, 1.0],
                              dy=[0.1, 0.9, -2.5, 0.0, 1.5, -1.0])
    out = oracle.reduce_set(fs, interp=interp)
    want = (1500.0 - 1000.0 - np.float64(np.float32(0.05)) * 60.0) / np.float64(np.float32(0.8))
    inner = np.s_[4:-4, 4:-4]
    np.testing.assert_allclose(out["mean"][inner], want, rtol=1e-12)
    np.testing.assert_allclose(out["median"][inner], want, rtol=1e-12)
    assert (out["nkept"][inner] == 6).all()


@pytest.mark.parametrize("interp", ["nearest", "bilinear", "spline3"])
def test_reduce_set_per_frame_exposure_and_flat_normalisation(interp):
    """Worked by hand.  Three constant frames of raw 1500, 1600, 1700 ADU with
    exposures 10, 60 and 100 s, bias 1000 ADU, dark rate 0.5 ADU/s, zero
    offsets (every interpolation is the identity).  Each frame's dark is its
    own exposure times the rate (Sec. 2.1 dark subtraction): raw - bias - dark
    = 495, 570, 650 ADU.  Three samples cannot be clipped at kappa 3
    (Samuelson), so the mean is 1715 / 3 and the median 570, each divided by
    the pixel's flat."""
    W, H = 6, 5
    raw = np.empty((3, H, W), np.uint16)
    raw[0], raw[1], raw[2] = 1500, 1600, 1700
    bias = np.full((H, W), 1000.0, np.float32)
    dark = np.full((H, W), 0.5, np.float32)
    t = np.array([10.0, 60.0, 100.0], np.float32)
    zero = np.zeros(3)
    # flat 0.5 everywhere: 990, 1140, 1300 -> median 1140, mean 3430 / 3
    fs = synth.FrameSet(raw=raw, bias=bias, dark=dark, flat=np.full((H, W), 0.5, np.float32),
                        exptime=t, dx=zero, dy=zero)
    out = oracle.reduce_set(fs, interp=interp)
    np.testing.assert_allclose(out["median"], 1140.0, rtol=1e-12)
    np.testing.assert_allclose(out["mean"], 1143.3333333333333, rtol=1e-12)
    # flat 0.5 and 1.0 in alternate columns, normalised by its mean 0.75: the
    # flat becomes 2/3 and 4/3, so the values are 1.5x and 0.75x the
    # differences: median 855 and 427.5, mean 857.5 and 428.75
    flat = np.tile(np.array([0.5, 1.0], np.float32), (H, W // 2))
    fs = synth.FrameSet(raw=raw, bias=bias, dark=dark, flat=flat, exptime=t, dx=zero, dy=zero)
    out = oracle.reduce_set(fs, interp=interp, normalize_flat=True)
    np.testing.assert_allclose(out["median"][:, 0::2], 855.0, rtol=1e-12)
    np.testing.assert_allclose(out["median"][:, 1::2], 427.5, rtol=1e-12)
    np.testing.assert_allclose(out["mean"][:, 0::2], 857.5, rtol=1e-12)
    np.testing.assert_allclose(out["mean"][:, 1::2], 428.75, rtol=1e-12)
    assert (out["nkept"] == 3).all()


def test_reduce_set_composes_calibrate_shift_clip_median():
    fs = synth.make_set(40, 36, 7, 3.0, 9)
    full = oracle.reduce_set(fs, interp="bilinear", kappa=2.0, want_stack=True)
    # stack = calibrate + shift of each frame
    for k in range(fs.n):
        v = oracle.calibrate(fs.raw[k], fs.bias, fs.dark, fs.flat, fs.exptime[k])
        a, valid = oracle.shift(v, fs.dx[k], fs.dy[k], "bilinear")
        assert np.array_equal(valid, full["valid"][k])
        np.testing.assert_allclose(full["stack"][k][valid], a[valid], rtol=1e-15)
    comb = oracle.combine_stack(full["stack"], full["valid"], kappa=2.0)
    np.testing.assert_array_equal(comb["nkept"], full["nkept"])
    np.testing.assert_allclose(comb["mean"], full["mean"], rtol=1e-15, equal_nan=True)
    np.testing.assert_allclose(comb["median"], full["median"], rtol=1e-15, equal_nan=True)
    # pixel-list mode agrees with the full grid
    xs = np.array([0, 5, 39, 17], np.int32)
    ys = np.array([0, 35, 12, 20], np.int32)
    part = oracle.reduce_set(fs, interp="bilinear", kappa=2.0, pixels=(xs, ys))
    np.testing.assert_array_equal(part["mean"], full["mean"][ys, xs])
    np.testing.assert_array_equal(part["median"], full["median"][ys, xs])


def test_reduce_set_aligns_dithered_stars():
    """Offsets passed as the dither offsets line the scene up again: the
    median of the aligned stack is smoother than any single frame."""
    fs = synth.make_set(64, 64, 9, 4.0, 21, n_cr=0)
    out = oracle.reduce_set(fs, interp="spline3")
    v0 = oracle.calibrate(fs.raw[0], fs.bias, fs.dark, fs.flat, 60.0)
    sl = np.s_[8:-8, 8:-8]
    assert np.std(out["median"][sl]) < np.std(v0[sl])


# ------------------------------------------------- bad-pixel masking (Sec. 2.1)
def _valid(fs, interp, **kw):
    return oracle.reduce_set(fs, interp=interp, want_stack=True, **kw)["valid"][0]


def _geometric(fs, interp):
    return _valid(fs, interp)


def test_mask_footprint_bilinear_by_hand():
    """One bad pixel at (x=4, y=3) of a 9x7 frame: the invalid outputs are
    exactly those whose taps with non-zero weight reach it."""
    mask = np.zeros((7, 9), np.uint8)
    mask[3, 4] = 1
    cases = {
        (0.5, 0.5): [(3, 2), (4, 2), (3, 3), (4, 3)],   # 2x2 taps
        (0.0, 0.5): [(4, 2), (4, 3)],                   # fx = 0: one column
        (2.0, -1.0): [(2, 4)],                          # integer move
        (-0.25, 0.0): [(4, 3), (5, 3)],                 # floor(-0.25) = -1, fx = 0.75
    }
    for (dx, dy), bad in cases.items():
        fs = synth.make_const_set(9, 7, 1, 1500, 1000.0, 0.05, 0.8, 60.0, dx=[dx], dy=[dy])
        geo = _geometric(fs, "bilinear")
        got = _valid(fs, "bilinear", mask=mask)
        want = geo.copy()
        for x, y in bad:
            assert geo[y, x], (dx, dy, x, y)
            want[y, x] = False
        assert np.array_equal(got, want), (dx, dy)


def test_mask_footprint_nearest_and_spline_by_hand():
    mask = np.zeros((12, 12), np.uint8)
    mask[6, 5] = 1
    fs = synth.make_const_set(12, 12, 1, 1500, 1000.0, 0.05, 0.8, 60.0, dx=[0.75], dy=[0.0])
    # nearest: 0.75 rounds to +1, so output x = 4 reads the bad pixel
    got = _valid(fs, "nearest", mask=mask)
    want = _geometric(fs, "nearest")
    want[6, 4] = False
    assert np.array_equal(got, want)
    # spline, fx = 0.75, fy = 0: taps i0-1..i0+2 along x (all non-zero), and
    # j0-1..j0+1 along y (beta3(2) = 0 drops the fourth): 4 columns x 3 rows
    got = _valid(fs, "spline3", mask=mask)
    want = _geometric(fs, "spline3")
    for y in (5, 6, 7):
        for x in (3, 4, 5, 6):
            want[y, x] = False
    assert np.array_equal(got, want)


def test_saturation_level_marks_bad_pixels():
    fs = synth.make_const_set(9, 7, 1, 1500, 1000.0, 0.05, 0.8, 60.0, dx=[0.5], dy=[0.5])
    fs.raw[0, 3, 4] = 65535
    geo = _geometric(fs, "bilinear")
    got = _valid(fs, "bilinear", saturation=60000.0)
    want = geo.copy()
    for x, y in [(3, 2), (4, 2), (3, 3), (4, 3)]:
        want[y, x] = False
    assert np.array_equal(got, want)
    # a level above every raw value, or off, masks nothing
    assert np.array_equal(_valid(fs, "bilinear", saturation=70000.0), geo)
    assert np.array_equal(_valid(fs, "bilinear", saturation=0.0), geo)


def test_masked_sample_leaves_the_combine():
    """Three constant frames calibrating to 1000, 2000 and 4000 ADU (flat 0.5,
    no dark); the third is saturated at one pixel: that pixel combines the
    first two only."""
    fs = synth.make_const_set(6, 5, 3, 1500, 1000.0, 0.0, 0.5, 60.0)
    fs.raw[1] = 2000
    fs.raw[2] = 3000
    fs.raw[2, 2, 3] = 3001   # the one saturated sample (level 3001)
    out = oracle.reduce_set(fs, interp="nearest", saturation=3001.0)
    assert out["nkept"][2, 3] == 2
    assert out["median"][2, 3] == 1500.0
    assert out["mean"][2, 3] == 1500.0
    assert out["nkept"][0, 0] == 3
    assert out["median"][0, 0] == 2000.0



# ---------------------------------------------------- per-frame normalisation
def _frames(vals, W=2, H=2):
    """A set of frames with the given raw values, zero bias and dark, unit
    flat and no offsets (calibrated value = raw)."""
    raw = np.asarray(vals, np.uint16).reshape(len(vals), H, W)
    n = raw.shape[0]
    return synth.FrameSet(raw=raw, bias=np.zeros((H, W), np.float32),
                          dark=np.zeros((H, W), np.float32), flat=np.ones((H, W), np.float32),
                          exptime=np.full(n, 60.0, np.float32), dx=np.zeros(n), dy=np.zeros(n))


def test_frame_normalisation_worked_by_hand():
    # frame 0 = [[1, 2], [3, 4]] (mean 2.5), frame 1 = [[3, 4], [5, 6]] (mean 4.5)
    fs = _frames([[1, 2, 3, 4], [3, 4, 5, 6]])
    # zero: frame 1 gets 2.5 - 4.5 = -2 and equals frame 0; the mean is frame 0
    r = oracle.reduce_set(fs, frame_norm="zero")
    np.testing.assert_allclose(r["mean"], [[1, 2], [3, 4]], atol=1e-14)
    np.testing.assert_allclose(r["median"], [[1, 2], [3, 4]], atol=1e-14)
    # scale: frame 1 times 2.5 / 4.5 = 5/9: [[5/3, 20/9], [25/9, 30/9]];
    # two samples, nothing clipped: the mean of frame 0 and that
    r = oracle.reduce_set(fs, frame_norm="scale")
    want = (np.array([[1, 2], [3, 4]]) + np.array([[15, 20], [25, 30]]) / 9.0) / 2.0
    np.testing.assert_allclose(r["mean"], want, atol=1e-14)
    # none leaves the samples alone
    r = oracle.reduce_set(fs, frame_norm="none")
    np.testing.assert_allclose(r["mean"], [[2, 3], [4, 5]], atol=1e-14)


def test_frame_normalisation_levels_frames_of_different_levels():
    """Frames that differ only by a level (zero) or a gain (scale) become
    identical to frame 0, whatever the interpolation."""
    rng = np.random.default_rng(3)
    base = rng.integers(200, 2000, (6, 9)).astype(np.float64)
    for interp in ("bilinear", "nearest", "cubic", "spline3"):
        fs = _frames([base + d for d in (0, 150, -120, 400)], W=9, H=6)
        r = oracle.reduce_set(fs, interp=interp, frame_norm="zero", want_stack=True)
        np.testing.assert_allclose(r["stack"], np.broadcast_to(r["stack"][0], r["stack"].shape),
                                   atol=1e-9)
    fs = _frames([base * g for g in (1, 2, 4)], W=9, H=6)
    r = oracle.reduce_set(fs, frame_norm="scale", want_stack=True)
    np.testing.assert_allclose(r["stack"], np.broadcast_to(r["stack"][0], r["stack"].shape),
                               rtol=1e-14)
    np.testing.assert_allclose(r["mean"], base, rtol=1e-14)


def test_frame_normalisation_rejects_a_zero_frame_mean_for_scale():
    fs = _frames([[1, 2, 3, 4], [0, 0, 0, 0]])
    with pytest.raises(ValueError):
        oracle.reduce_set(fs, frame_norm="scale")
    oracle.reduce_set(fs, frame_norm="zero")  # an additive level needs no division

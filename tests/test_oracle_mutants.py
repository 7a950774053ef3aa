"""The oracle's pins catch plausible mistakes in the oracle.

Each case below plants one mistake in a copy of ``oracle/oracle.c`` (a
dropped term, a wrong sign, constant or index, a transposed operand, an
off-by-one bound, a loose inequality), compiles that copy, swaps it in for the
oracle and runs every pin of ``test_oracle.py`` against it.  At least one pin
must fail for every mistake; a mistake that no pin notices would leave the
oracle unchecked at that point.  The mistakes only change arithmetic and
stricter bounds, never make an access leave its array, so a broken copy fails
a comparison and cannot crash the test process.
"""
import inspect
import shutil

import pytest

import oracle
import test_oracle

# (name, text in oracle.c, the planted mistake); each text occurs once
MUTANTS = [
    # cubic B-spline basis (Sec. 3.1.1)
    ("beta3 inner piece drops the cubic term",
     "2.0 / 3.0 - a * a + 0.5 * a * a * a", "2.0 / 3.0 - a * a + 0.5 * a * a"),
    ("beta3 outer piece squared, not cubed", "return b * b * b / 6.0;", "return b * b / 6.0;"),
    # mirror boundary
    ("mirror period one sample short", "int64_t period = 2 * (N - 1);",
     "int64_t period = 2 * N - 1;"),
    # calibration (Sec. 2.1)
    ("calibration drops the dark current",
     "(r - (double)bias[m] - (double)dark[m] * t) / f;", "(r - (double)bias[m]) / f;"),
    ("calibration adds the dark current",
     "(r - (double)bias[m] - (double)dark[m] * t) / f;",
     "(r - (double)bias[m] + (double)dark[m] * t) / f;"),
    ("calibration multiplies by the flat",
     "(r - (double)bias[m] - (double)dark[m] * t) / f;",
     "(r - (double)bias[m] - (double)dark[m] * t) * f;"),
    ("on-demand calibration multiplies by the flat",
     "(r - (double)s->bias[m] - (double)s->dark[m] * s->t) / f;",
     "(r - (double)s->bias[m] - (double)s->dark[m] * s->t) * f;"),
    ("flat normalisation inverted", "double f = (double)flat[m] / flat_norm;",
     "double f = (double)flat[m] * flat_norm;"),
    ("flat mean over one row's count", "return s / ((double)W * (double)H);",
     "return s / (double)W;"),
    # spline system (Sec. 3.2.1)
    ("spline system without the mirror doubling at the first row",
     "((i == 0) ? 2.0 / 6.0 : 1.0 / 6.0)", "((i == 0) ? 1.0 / 6.0 : 1.0 / 6.0)"),
    ("spline system without the mirror doubling at the last row",
     "((i == N - 1) ? 2.0 / 6.0 : 1.0 / 6.0)", "((i == N - 1) ? 1.0 / 6.0 : 1.0 / 6.0)"),
    ("spline system diagonal 1 instead of 4/6", "double diag = 4.0 / 6.0;",
     "double diag = 1.0;"),
    ("spline back substitution adds", "c[(int64_t)i * cstride] = rp[i] - cp[i] *",
     "c[(int64_t)i * cstride] = rp[i] + cp[i] *"),
    ("spline solved along rows only",
     "    oracle_spline_solve_line(tmp, 1, col, 1, H, work);\n",
     "    for (int y = 0; y < H; ++y) col[y] = tmp[y];\n"),
    # resampling
    ("offset applied with the wrong sign", "int64_t i0 = (int64_t)x + (int64_t)fdx;",
     "int64_t i0 = (int64_t)x - (int64_t)fdx;"),
    ("fractional part with the wrong sign", "double fx = dx - fdx, fy = dy - fdy;",
     "double fx = fdx - dx, fy = dy - fdy;"),
    ("nearest rounds halves down", "return (i0 >= 0) ? i0 + 1 : i0;", "return i0;"),
    ("validity drops the last column for integer positions",
     "if (fr == 0.0) return i0 <= N - 1;", "if (fr == 0.0) return i0 < N - 1;"),
    ("spline horizontal weights mirrored", "double w = oracle_bspline3(fx + 1.0 - p) * wyq;",
     "double w = oracle_bspline3(fx - 1.0 + p) * wyq;"),
    ("spline vertical weights from the x fraction",
     "double wyq = oracle_bspline3(fy + 1.0 - q);", "double wyq = oracle_bspline3(fx + 1.0 - q);"),
    # bad pixels (Sec. 2.1)
    ("bilinear ignores bad pixels", "        if (src_bad(s, i0 + p, j0 + q)) return 0;\n", ""),
    ("saturation only above the level", ">= s->saturation", "> s->saturation"),
    # Keys cubic convolution
    ("keys a = +1/2", "const double a = -0.5;", "const double a = 0.5;"),
    ("keys inner branch squared term", "return 1.0 - (a + 3.0) * x * x + (a + 2.0) * x * x * x;",
     "return 1.0 - (a + 2.0) * x * x + (a + 2.0) * x * x * x;"),
    ("keys outer branch", "if (x < 2.0) return a * (x - 1.0) * (x - 2.0) * (x - 2.0);",
     "if (x < 2.0) return a * (x - 1.0) * (x - 1.0) * (x - 2.0);"),
    ("keys taps shifted", "double wxp = oracle_keys(fx + 1.0 - p);",
     "double wxp = oracle_keys(fx - p);"),
    ("keys validity ignores the last tap", "return i0 - 1 >= 0 && i0 + 2 <= N - 1;",
     "return i0 - 1 >= 0 && i0 + 1 <= N - 1;"),
    # per-frame normalisation
    ("normalisation zero sign", "nz[k] = m[0] - m[k];", "nz[k] = m[k] - m[0];"),
    ("normalisation scale inverted", "ns[k] = m[0] / m[k];", "ns[k] = m[k] / m[0];"),
    ("normalisation statistic not divided by the pixel count", "m[k] = sum / (double)P;",
     "m[k] = sum;"),
    # sigma clip and median
    ("clip rejects at the threshold", "if (fabs(d) > thr) {", "if (fabs(d) >= thr) {"),
    ("clip ignores ddof", "double sigma = sqrt(ss / (double)(m - p->ddof));",
     "double sigma = sqrt(ss / (double)m);"),
    ("clip swaps the lower and upper kappa", "(d < 0.0 ? p->kappa_lo : p->kappa_hi)",
     "(d < 0.0 ? p->kappa_hi : p->kappa_lo)"),
    ("clip runs one pass too many", "for (int it = 0; it < p->max_iter; ++it) {",
     "for (int it = 0; it <= p->max_iter; ++it) {"),
    ("clip ignores the median centre", "if (p->center == 1) {", "if (p->center == 2) {"),
    ("clipped mean over all samples", "*mean = (m == 0) ? NAN : s / m;",
     "*mean = (m == 0) ? NAN : s / n;"),
    ("median of an even count is the upper middle value",
     "return 0.5 * (buf[(m - 1) / 2] + buf[m / 2]);", "return buf[m / 2];"),
    # the whole set
    ("every frame takes the first frame's exposure time", "src[k].t = exptime[k];",
     "src[k].t = exptime[0];"),
    ("spline frames take the first frame's exposure time",
     "master_pitch,\n                       exptime[k], flat_norm, v);",
     "master_pitch,\n                       exptime[0], flat_norm, v);"),
    ("the set ignores flat normalisation",
     "double flat_norm = normalize_flat ? oracle_mean_f32(flat, master_pitch, W, H) : 1.0;",
     "double flat_norm = 1.0;"),
    ("sampled pixels swap x and y", "int x = npix > 0 ? px[o] : (int)(o % W);",
     "int x = npix > 0 ? py[o] : (int)(o % W);"),
    ("each frame sampled at the first frame's offset",
     "sample_src(&src[k], W, H, x, y, dx[k], dy[k], interp, &a);",
     "sample_src(&src[k], W, H, x, y, dx[0], dy[k], interp, &a);"),
    # validity and masks
    ("clip counts invalid samples", "alive[k] = valid[k] ? 1 : 0;", "alive[k] = 1;"),
    ("median counts invalid samples", "    if (valid[k]) buf[m++] = x[k];\n",
     "    buf[m++] = x[k];\n"),
    ("stack combine ignores validity", "ok[k] = valid[(int64_t)k * P + o];", "ok[k] = 1;"),
    ("nearest ignores bad pixels", "    if (src_bad(s, i, j)) return 0;\n", ""),
    ("spline ignores bad pixels",
     "if (w != 0.0 && src_bad(s, oracle_mirror(i, W), oracle_mirror(j, H))) return 0;", ""),
    ("clip margin not in units of sigma", "double mg = dist / sigma;", "double mg = dist;"),
    ("clip margin in data units divided by sigma",
     "if (dist < margin_adu) margin_adu = dist;", "if (dist / sigma < margin_adu) margin_adu = dist / sigma;"),
    ("clip margin in data units from the signed deviation",
     "double dist = fabs(fabs(d) - thr);", "double dist = fabs(d - thr);"),
    ("shift marks every sample valid", "valid[(int64_t)y * W + x] = (uint8_t)ok;",
     "valid[(int64_t)y * W + x] = 1;"),
    ("every spline frame takes the first frame's coefficients",
     "src[k].f = coef + (int64_t)k * P;", "src[k].f = coef;"),
    ("median leaves out samples far from the clipped mean", "        if (ok[k]) tmp[m++] = s[k];\n",
     "        if (ok[k] && fabs(s[k] - mu) <= 3.0 * fabs(mu)) tmp[m++] = s[k];\n"),
]


def _pin_calls():
    """Every pin of test_oracle.py with each of its parameter sets."""
    calls = []
    for name, fn in inspect.getmembers(test_oracle, inspect.isfunction):
        if not name.startswith("test_"):
            continue
        combos = [{}]
        for mark in getattr(fn, "pytestmark", []):
            if mark.name != "parametrize":
                continue
            names = [a.strip() for a in mark.args[0].split(",")]
            combos = [dict(c, **dict(zip(names, v if len(names) > 1 else (v,))))
                      for c in combos for v in mark.args[1]]
        calls += [(name, fn, kw) for kw in combos]
    return calls


PINS = _pin_calls()


def _failing_pins():
    failed = []
    for name, fn, kw in PINS:
        try:
            fn(**kw)
        except Exception:  # an assertion or a rejected call: the pin noticed
            failed.append(f"{name}{kw or ''}")
    return failed


def test_pins_pass_on_the_oracle_as_written():
    assert len(PINS) >= 40
    assert _failing_pins() == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_a_planted_mistake_fails_a_pin(name, old, new, tmp_path, monkeypatch):
    with open(oracle._SRC) as f:
        src = f.read()
    assert src.count(old) == 1, "the planted mistake no longer matches oracle.c"
    path = tmp_path / "oracle.c"
    path.write_text(src.replace(old, new))
    shutil.copy(oracle._SRC.replace("oracle.c", "oracle.h"), tmp_path / "oracle.h")
    broken = oracle.load(oracle.compile_library(str(path), str(tmp_path / "liboracle.so")))
    monkeypatch.setattr(oracle, "_lib", broken)
    assert _failing_pins(), f"no pin notices: {name}"

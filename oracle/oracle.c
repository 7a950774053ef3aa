/*
 * oracle.c -- plain FP64 CPU oracle of the image-reduction hot path.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the package smoke check
 * and the benchmark's CPU-baseline leg, never by the product path.  It shares
 * no code with the CUDA path.  Every step is the plain definition, in double
 * precision, in the order the paper describes the pipeline:
 *
 *   Sec. 2.1: overscan cutout, bias subtraction, dark subtraction, flat
 *             fielding, bad-pixel masking, alignment, co-adding; the 16-bit
 *             integers become floating point at bias subtraction.
 *   Sec. 2.1 / 2.2: alignment by "bicubic-spline interpolation", co-adding by
 *             a sigma-clipped mean.
 *   Sec. 3.1.1: cubic-spline interpolation reproduces cubic B-spline basis
 *             functions exactly (the basis is beta3 below).
 *   Sec. 3.2.1: the spline needs one tridiagonal linear system per row and
 *             per column of the image; it is solved here by banded Gaussian
 *             elimination (the Thomas algorithm), O(N) per line.
 *
 * Readings where the paper is silent (dark scaling with exposure time, spline
 * boundary condition, offset sign, validity at the frame edges, clip centre,
 * sigma estimator, strict inequality, median for even counts) are fixed as:
 *   dark master is a rate (ADU/s) scaled by each frame's exposure time;
 *   mirror (whole-sample symmetric) boundary for the spline;
 *   output pixel (x, y) samples frame k at (x + dx_k, y + dy_k), the offset
 *   split as dx = ix + fx with ix = floor(dx), fx in [0, 1);
 *   a sample is valid iff every tap with non-zero weight lies in the frame
 *   (nearest, bilinear) or the source position lies in [0,W-1]x[0,H-1]
 *   (spline; the same integer condition);
 *   clip around the mean (or median), population sigma (ddof 0), strict '>',
 *   cumulative rejection, stop when nothing is rejected or sigma = 0;
 *   median of all valid samples before clipping, even count -> mean of the two
 *   middle values.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

double oracle_bspline3(double t) {
  double a = fabs(t);
  if (a < 1.0) return 2.0 / 3.0 - a * a + 0.5 * a * a * a;
  if (a < 2.0) {
    double b = 2.0 - a;
    return b * b * b / 6.0;
  }
  return 0.0;
}

double oracle_keys(double t) {
  const double a = -0.5;
  double x = fabs(t);
  if (x <= 1.0) return 1.0 - (a + 3.0) * x * x + (a + 2.0) * x * x * x;
  if (x < 2.0) return a * (x - 1.0) * (x - 2.0) * (x - 2.0);
  return 0.0;
}

int64_t oracle_mirror(int64_t i, int64_t N) {
  if (N <= 1) return 0;
  int64_t period = 2 * (N - 1);
  int64_t r = i % period;
  if (r < 0) r += period;
  if (r >= N) r = period - r;
  return r;
}

double oracle_mean_f32(const float* a, int64_t pitch, int W, int H) {
  double s = 0.0;
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) s += (double)a[(int64_t)y * pitch + x];
  return s / ((double)W * (double)H);
}

/* Sec. 2.1: v = (raw - bias - dark * t) / flat, the flat optionally divided by
 * its own mean first (flat_norm = 1 leaves it unchanged). */
void oracle_calibrate(const uint16_t* raw, int64_t raw_pitch, int W, int H,
                      const float* bias, const float* dark, const float* flat,
                      int64_t master_pitch, double t, double flat_norm, double* v) {
  for (int y = 0; y < H; ++y) {
    for (int x = 0; x < W; ++x) {
      int64_t m = (int64_t)y * master_pitch + x;
      double r = (double)raw[(int64_t)y * raw_pitch + x];
      double f = (double)flat[m] / flat_norm;
      v[(int64_t)y * W + x] = (r - (double)bias[m] - (double)dark[m] * t) / f;
    }
  }
}

/* The interpolation condition sum_i c[i] beta3(j - i) = v[j] at every sample j
 * is (c[j-1] + 4 c[j] + c[j+1]) / 6 = v[j].  With the mirror extension
 * c[-1] = c[1] and c[N] = c[N-2], the first and last rows become
 * (4 c[0] + 2 c[1]) / 6 = v[0] and (2 c[N-2] + 4 c[N-1]) / 6 = v[N-1]:
 * a tridiagonal system, eliminated forward and substituted back. */
void oracle_spline_solve_line(const double* v, int64_t vstride, double* c, int64_t cstride,
                              int N, double* work) {
  if (N == 1) {  /* every mirrored index is 0: (c + 4c + c)/6 = v */
    c[0] = v[0];
    return;
  }
  double* cp = work;      /* modified super-diagonal */
  double* rp = work + N;  /* modified right-hand side */
  for (int i = 0; i < N; ++i) {
    double sub = (i == 0) ? 0.0 : ((i == N - 1) ? 2.0 / 6.0 : 1.0 / 6.0);
    double diag = 4.0 / 6.0;
    double sup = (i == N - 1) ? 0.0 : ((i == 0) ? 2.0 / 6.0 : 1.0 / 6.0);
    double rhs = v[(int64_t)i * vstride];
    if (i == 0) {
      cp[0] = sup / diag;
      rp[0] = rhs / diag;
    } else {
      double den = diag - sub * cp[i - 1];
      cp[i] = sup / den;
      rp[i] = (rhs - sub * rp[i - 1]) / den;
    }
  }
  c[(int64_t)(N - 1) * cstride] = rp[N - 1];
  for (int i = N - 2; i >= 0; --i)
    c[(int64_t)i * cstride] = rp[i] - cp[i] * c[(int64_t)(i + 1) * cstride];
}

/* Separable 2-D system: (B (x) B) c = v, so rows are solved, then columns. */
void oracle_spline_coeffs(const double* v, int W, int H, double* c) {
  int nmax = W > H ? W : H;
  double* work = (double*)malloc(sizeof(double) * 2 * (size_t)nmax);
  double* tmp = (double*)malloc(sizeof(double) * (size_t)nmax);
  double* col = (double*)malloc(sizeof(double) * (size_t)nmax);
  for (int y = 0; y < H; ++y)
    oracle_spline_solve_line(v + (int64_t)y * W, 1, c + (int64_t)y * W, 1, W, work);
  for (int x = 0; x < W; ++x) {
    for (int y = 0; y < H; ++y) tmp[y] = c[(int64_t)y * W + x];
    oracle_spline_solve_line(tmp, 1, col, 1, H, work);
    for (int y = 0; y < H; ++y) c[(int64_t)y * W + x] = col[y];
  }
  free(work);
  free(tmp);
  free(col);
}

/* Frame data source: a full FP64 frame, or raw + masters calibrated on demand;
 * plus the bad-pixel definition (Sec. 2.1 bad-pixel masking): a source pixel
 * is bad when the mask master marks it or its raw value reaches the
 * saturation level (mask NULL / saturation <= 0: no such test). */
typedef struct {
  const double* f;
  const uint16_t* raw;
  int64_t raw_pitch;
  const float *bias, *dark, *flat;
  int64_t master_pitch;
  double t, flat_norm;
  const uint8_t* mask;
  int64_t mask_pitch;
  double saturation;
} frame_src;

static int src_bad(const frame_src* s, int64_t i, int64_t j) {
  if (s->mask && s->mask[j * s->mask_pitch + i]) return 1;
  if (s->saturation > 0.0 && s->raw && (double)s->raw[j * s->raw_pitch + i] >= s->saturation)
    return 1;
  return 0;
}

static double src_value(const frame_src* s, int W, int64_t i, int64_t j) {
  if (s->f) return s->f[j * W + i];
  int64_t m = j * s->master_pitch + i;
  double r = (double)s->raw[j * s->raw_pitch + i];
  double f = (double)s->flat[m] / s->flat_norm;
  return (r - (double)s->bias[m] - (double)s->dark[m] * s->t) / f;
}

/* Along one axis: the source position is i0 + fr with i0 = p + floor(d) and
 * fr = d - floor(d) in [0, 1).  A tap is needed iff its weight is non-zero. */
static int axis_valid_linear(int64_t i0, double fr, int64_t N) {
  if (i0 < 0) return 0;
  if (fr == 0.0) return i0 <= N - 1;
  return i0 + 1 <= N - 1;
}

/* Keys' cubic convolution: taps i0-1 .. i0+2 with weights W(fr + 1 - p); for
 * fr = 0 only the tap at i0 has non-zero weight. */
static int axis_valid_keys(int64_t i0, double fr, int64_t N) {
  if (fr == 0.0) return i0 >= 0 && i0 <= N - 1;
  return i0 - 1 >= 0 && i0 + 2 <= N - 1;
}

/* Nearest integer to i0 + fr, halves rounded away from zero. */
static int64_t axis_nearest(int64_t i0, double fr) {
  if (fr < 0.5) return i0;
  if (fr > 0.5) return i0 + 1;
  return (i0 >= 0) ? i0 + 1 : i0; /* i0 + 0.5 > 0 iff i0 >= 0 */
}

static int sample_src(const frame_src* s, int W, int H, int x, int y, double dx, double dy,
                      int interp, double* a) {
  double fdx = floor(dx), fdy = floor(dy);
  double fx = dx - fdx, fy = dy - fdy;
  int64_t i0 = (int64_t)x + (int64_t)fdx;
  int64_t j0 = (int64_t)y + (int64_t)fdy;
  if (interp == ORACLE_NEAREST) {
    int64_t i = axis_nearest(i0, fx), j = axis_nearest(j0, fy);
    if (i < 0 || i > W - 1 || j < 0 || j > H - 1) return 0;
    if (src_bad(s, i, j)) return 0;
    *a = src_value(s, W, i, j);
    return 1;
  }
  if (interp == ORACLE_CUBIC) {
    /* every tap with non-zero weight inside the frame and not bad */
    if (!axis_valid_keys(i0, fx, W) || !axis_valid_keys(j0, fy, H)) return 0;
    double acc = 0.0;
    for (int q = 0; q < 4; ++q) {
      double wyq = oracle_keys(fy + 1.0 - q);
      if (wyq == 0.0) continue; /* zero-weight taps are not read */
      for (int p = 0; p < 4; ++p) {
        double wxp = oracle_keys(fx + 1.0 - p);
        if (wxp == 0.0) continue;
        if (src_bad(s, i0 - 1 + p, j0 - 1 + q)) return 0;
        acc += wxp * wyq * src_value(s, W, i0 - 1 + p, j0 - 1 + q);
      }
    }
    *a = acc;
    return 1;
  }
  if (!axis_valid_linear(i0, fx, W) || !axis_valid_linear(j0, fy, H)) return 0;
  if (interp == ORACLE_BILINEAR) {
    double wx[2] = {1.0 - fx, fx}, wy[2] = {1.0 - fy, fy};
    double acc = 0.0;
    for (int q = 0; q < 2; ++q)
      for (int p = 0; p < 2; ++p) {
        double w = wx[p] * wy[q];
        if (w == 0.0) continue; /* zero-weight taps are not read */
        if (src_bad(s, i0 + p, j0 + q)) return 0;
        acc += w * src_value(s, W, i0 + p, j0 + q);
      }
    *a = acc;
    return 1;
  }
  /* cubic spline: a = sum_{i,j} c[i,j] beta3(xs - i) beta3(ys - j) over the
   * four taps around the position, coefficients mirrored outside the frame;
   * a tap with non-zero weight on a bad pixel (after mirroring) invalidates
   * the sample */
  double acc = 0.0;
  for (int q = 0; q < 4; ++q) {
    int64_t j = j0 - 1 + q;
    double wyq = oracle_bspline3(fy + 1.0 - q);
    for (int p = 0; p < 4; ++p) {
      int64_t i = i0 - 1 + p;
      double w = oracle_bspline3(fx + 1.0 - p) * wyq;
      if (w != 0.0 && src_bad(s, oracle_mirror(i, W), oracle_mirror(j, H))) return 0;
      acc += w * src_value(s, W, oracle_mirror(i, W), oracle_mirror(j, H));
    }
  }
  *a = acc;
  return 1;
}

int oracle_sample(const double* f, int W, int H, int x, int y, double dx, double dy,
                  int interp, double* a) {
  frame_src s;
  memset(&s, 0, sizeof(s));
  s.f = f;
  return sample_src(&s, W, H, x, y, dx, dy, interp, a);
}

void oracle_shift(const double* v, int W, int H, double dx, double dy, int interp,
                  double* a, uint8_t* valid) {
  const double* f = v;
  double* coef = NULL;
  if (interp == ORACLE_SPLINE3) {
    coef = (double*)malloc(sizeof(double) * (size_t)W * (size_t)H);
    oracle_spline_coeffs(v, W, H, coef);
    f = coef;
  }
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      double val = 0.0;
      int ok = oracle_sample(f, W, H, x, y, dx, dy, interp, &val);
      a[(int64_t)y * W + x] = ok ? val : 0.0;
      valid[(int64_t)y * W + x] = (uint8_t)ok;
    }
  free(coef);
}

static int cmp_double(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return (x > y) - (x < y);
}

static double median_of(double* buf, int m) {
  qsort(buf, (size_t)m, sizeof(double), cmp_double);
  return 0.5 * (buf[(m - 1) / 2] + buf[m / 2]);
}

double oracle_median(const double* x, const uint8_t* valid, int n) {
  double* buf = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  int m = 0;
  for (int k = 0; k < n; ++k)
    if (valid[k]) buf[m++] = x[k];
  double r = (m == 0) ? NAN : median_of(buf, m);
  free(buf);
  return r;
}

void oracle_clip(const double* x, const uint8_t* valid, int n, const oracle_clip_params* p,
                 double* mean, int* nkept, uint8_t* rejected, double* min_margin,
                 double* min_margin_adu) {
  uint8_t* alive = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
  uint8_t* rej = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
  double* buf = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double margin = INFINITY, margin_adu = INFINITY;
  for (int k = 0; k < n; ++k) {
    alive[k] = valid[k] ? 1 : 0;
    if (rejected) rejected[k] = 0;
  }
  for (int it = 0; it < p->max_iter; ++it) {
    int m = 0;
    for (int k = 0; k < n; ++k) m += alive[k];
    if (m == 0 || m - p->ddof <= 0) break;
    double mu;
    if (p->center == 1) {
      int q = 0;
      for (int k = 0; k < n; ++k)
        if (alive[k]) buf[q++] = x[k];
      mu = median_of(buf, q);
    } else {
      double s = 0.0;
      for (int k = 0; k < n; ++k)
        if (alive[k]) s += x[k];
      mu = s / m;
    }
    double ss = 0.0;
    for (int k = 0; k < n; ++k)
      if (alive[k]) ss += (x[k] - mu) * (x[k] - mu);
    double sigma = sqrt(ss / (double)(m - p->ddof));
    if (sigma == 0.0) break;
    int nrej = 0;
    for (int k = 0; k < n; ++k) {
      rej[k] = 0;
      if (!alive[k]) continue;
      double d = x[k] - mu;
      double thr = (d < 0.0 ? p->kappa_lo : p->kappa_hi) * sigma;
      double dist = fabs(fabs(d) - thr);  /* distance to the threshold, data units */
      if (dist < margin_adu) margin_adu = dist;
      double mg = dist / sigma;
      if (mg < margin) margin = mg;
      if (fabs(d) > thr) {
        rej[k] = 1;
        ++nrej;
      }
    }
    if (nrej == 0) break;
    for (int k = 0; k < n; ++k)
      if (rej[k]) {
        alive[k] = 0;
        if (rejected) rejected[k] = 1;
      }
  }
  int m = 0;
  double s = 0.0;
  for (int k = 0; k < n; ++k)
    if (alive[k]) {
      s += x[k];
      ++m;
    }
  *mean = (m == 0) ? NAN : s / m;
  *nkept = m;
  if (min_margin) *min_margin = margin;
  if (min_margin_adu) *min_margin_adu = margin_adu;
  free(alive);
  free(rej);
  free(buf);
}

int oracle_reduce_set(const uint16_t* raw, int64_t raw_pitch, int64_t frame_stride,
                      int W, int H, int n,
                      const float* bias, const float* dark, const float* flat,
                      int64_t master_pitch, const double* exptime,
                      const double* dx, const double* dy, int interp, int normalize_flat,
                      const oracle_clip_params* clip, int nthreads,
                      int64_t npix, const int32_t* px, const int32_t* py,
                      double* mean, double* median, int32_t* nkept, double* min_margin,
                      double* min_margin_adu, double* stack, uint8_t* valid) {
  return oracle_reduce_set_masked(raw, raw_pitch, frame_stride, W, H, n, bias, dark, flat,
                                  master_pitch, exptime, dx, dy, interp, normalize_flat, NULL, 0,
                                  0.0, clip, nthreads, npix, px, py, mean, median, nkept,
                                  min_margin, min_margin_adu, stack, valid, ORACLE_NORM_NONE);
}

int oracle_reduce_set_masked(const uint16_t* raw, int64_t raw_pitch, int64_t frame_stride,
                             int W, int H, int n,
                             const float* bias, const float* dark, const float* flat,
                             int64_t master_pitch, const double* exptime,
                             const double* dx, const double* dy, int interp, int normalize_flat,
                             const uint8_t* mask, int64_t mask_pitch, double saturation,
                             const oracle_clip_params* clip, int nthreads,
                             int64_t npix, const int32_t* px, const int32_t* py,
                             double* mean, double* median, int32_t* nkept, double* min_margin,
                             double* min_margin_adu, double* stack, uint8_t* valid,
                             int frame_norm) {
  if (W < 1 || H < 1 || n < 1 || raw_pitch < W || master_pitch < W) return 1;
  if (frame_norm < ORACLE_NORM_NONE || frame_norm > ORACLE_NORM_SCALE) return 1;
  if (interp < ORACLE_NEAREST || interp > ORACLE_CUBIC) return 1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  double flat_norm = normalize_flat ? oracle_mean_f32(flat, master_pitch, W, H) : 1.0;
  int64_t P = (int64_t)W * H;
  double* coef = NULL;
  frame_src* src = (frame_src*)calloc((size_t)n, sizeof(frame_src));
  for (int k = 0; k < n; ++k) {
    src[k].raw = raw + (int64_t)k * frame_stride;
    src[k].raw_pitch = raw_pitch;
    src[k].bias = bias;
    src[k].dark = dark;
    src[k].flat = flat;
    src[k].master_pitch = master_pitch;
    src[k].t = exptime[k];
    src[k].flat_norm = flat_norm;
    src[k].mask = mask;
    src[k].mask_pitch = mask_pitch;
    src[k].saturation = saturation;
  }
  if (interp == ORACLE_SPLINE3) {
    /* the spline couples whole rows and columns: solve every frame fully */
    coef = (double*)malloc(sizeof(double) * (size_t)P * (size_t)n);
#pragma omp parallel for schedule(dynamic, 1) if (nthreads > 1)
    for (int k = 0; k < n; ++k) {
      double* v = (double*)malloc(sizeof(double) * (size_t)P);
      oracle_calibrate(src[k].raw, raw_pitch, W, H, bias, dark, flat, master_pitch,
                       exptime[k], flat_norm, v);
      oracle_spline_coeffs(v, W, H, coef + (int64_t)k * P);
      free(v);
    }
    for (int k = 0; k < n; ++k) src[k].f = coef + (int64_t)k * P;
  }
  /* per-frame normalisation before the combine: the frame statistic is the
   * mean of the calibrated frame over all its pixels, the reference frame 0;
   * zero: x + (m_0 - m_k), scale: x * (m_0 / m_k) */
  double* nz = (double*)calloc((size_t)n, sizeof(double));
  double* ns = (double*)malloc(sizeof(double) * (size_t)n);
  for (int k = 0; k < n; ++k) ns[k] = 1.0;
  if (frame_norm != ORACLE_NORM_NONE) {
    double* m = (double*)malloc(sizeof(double) * (size_t)n);
    double* v = (double*)malloc(sizeof(double) * (size_t)P);
    for (int k = 0; k < n; ++k) {
      oracle_calibrate(src[k].raw, raw_pitch, W, H, bias, dark, flat, master_pitch, src[k].t,
                       flat_norm, v);
      double sum = 0.0;
      for (int64_t i = 0; i < P; ++i) sum += v[i];
      m[k] = sum / (double)P;
    }
    int bad = 0;
    for (int k = 0; k < n; ++k) {
      if (frame_norm == ORACLE_NORM_ZERO) {
        nz[k] = m[0] - m[k];
      } else {
        if (!(m[k] != 0.0) || !isfinite(m[k])) bad = 1;
        ns[k] = m[0] / m[k];
      }
    }
    free(v);
    free(m);
    if (bad) {
      free(nz);
      free(ns);
      free(coef);
      free(src);
      return 2;
    }
  }
  int64_t nout = npix > 0 ? npix : P;
#pragma omp parallel if (nthreads > 1)
  {
    double* s = (double*)malloc(sizeof(double) * (size_t)n);
    double* tmp = (double*)malloc(sizeof(double) * (size_t)n);
    uint8_t* ok = (uint8_t*)malloc((size_t)n);
#pragma omp for schedule(dynamic, 256)
    for (int64_t o = 0; o < nout; ++o) {
      int x = npix > 0 ? px[o] : (int)(o % W);
      int y = npix > 0 ? py[o] : (int)(o / W);
      for (int k = 0; k < n; ++k) {
        double a = 0.0;
        ok[k] = (uint8_t)sample_src(&src[k], W, H, x, y, dx[k], dy[k], interp, &a);
        if (frame_norm == ORACLE_NORM_ZERO) a += nz[k];
        if (frame_norm == ORACLE_NORM_SCALE) a *= ns[k];
        s[k] = ok[k] ? a : 0.0;
        if (stack && npix <= 0) stack[(int64_t)k * P + o] = s[k];
        if (valid && npix <= 0) valid[(int64_t)k * P + o] = ok[k];
      }
      int kept = 0;
      double mg = INFINITY, mga = INFINITY, mu = 0.0;
      oracle_clip(s, ok, n, clip, &mu, &kept, NULL, &mg, &mga);
      mean[o] = mu;
      if (nkept) nkept[o] = kept;
      if (min_margin) min_margin[o] = mg;
      if (min_margin_adu) min_margin_adu[o] = mga;
      int m = 0;
      for (int k = 0; k < n; ++k)
        if (ok[k]) tmp[m++] = s[k];
      median[o] = (m == 0) ? NAN : median_of(tmp, m);
    }
    free(s);
    free(tmp);
    free(ok);
  }
  free(nz);
  free(ns);
  free(coef);
  free(src);
  return 0;
}

void oracle_combine_stack(const double* stack, const uint8_t* valid, int n, int64_t P,
                          const oracle_clip_params* clip, int nthreads, double* mean,
                          double* median, int32_t* nkept, double* min_margin,
                          double* min_margin_adu, uint8_t* rejected) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel if (nthreads > 1)
  {
    double* x = (double*)malloc(sizeof(double) * (size_t)n);
    uint8_t* ok = (uint8_t*)malloc((size_t)n);
    uint8_t* rej = (uint8_t*)malloc((size_t)n);
#pragma omp for schedule(dynamic, 1024)
    for (int64_t o = 0; o < P; ++o) {
      for (int k = 0; k < n; ++k) {
        x[k] = stack[(int64_t)k * P + o];
        ok[k] = valid[(int64_t)k * P + o];
      }
      int kept = 0;
      double mg = INFINITY, mga = INFINITY, mu = 0.0;
      oracle_clip(x, ok, n, clip, &mu, &kept, rej, &mg, &mga);
      mean[o] = mu;
      nkept[o] = kept;
      min_margin[o] = mg;
      if (min_margin_adu) min_margin_adu[o] = mga;
      median[o] = oracle_median(x, ok, n);
      if (rejected)
        for (int k = 0; k < n; ++k) rejected[(int64_t)k * P + o] = rej[k];
    }
    free(x);
    free(ok);
    free(rej);
  }
}

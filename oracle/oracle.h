/*
 * oracle.h -- plain FP64 CPU oracle of the image-reduction hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * What it computes (all arithmetic in double precision):
 *   calibration   v = (raw - bias - dark*t) / flat           (Sec. 2.1, Sec. 2.2)
 *   resampling    a(x,y) = v(x+dx, y+dy), nearest / bilinear / cubic spline
 *                 (Sec. 2.1 "bicubic-spline interpolation"; Sec. 3.1.1; Sec. 3.2.1)
 *   combination   iterative sigma-clipped mean (Sec. 2.1) and median.
 */
#ifndef IRP_ORACLE_H
#define IRP_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_NEAREST = 0, ORACLE_BILINEAR = 1, ORACLE_SPLINE3 = 2, ORACLE_CUBIC = 3 };

/* Per-frame normalisation before the combine (a combine variant): the
 * statistic of frame k is m_k, the mean of its calibrated values over the
 * whole frame, and frame 0 is the reference.  ZERO adds m_0 - m_k to every
 * sample of frame k, SCALE multiplies it by m_0 / m_k. */
enum { ORACLE_NORM_NONE = 0, ORACLE_NORM_ZERO = 1, ORACLE_NORM_SCALE = 2 };

typedef struct {
  double kappa_lo;   /* reject x if (mu - x) >  kappa_lo * sigma            */
  double kappa_hi;   /* reject x if (x - mu) >  kappa_hi * sigma            */
  int max_iter;      /* at most this many rejection passes                  */
  int center;        /* 0: clip around the mean, 1: around the median       */
  int ddof;          /* sigma^2 = sum (x-mu)^2 / (m - ddof)                 */
} oracle_clip_params;

/* Cubic B-spline basis function beta3(t) (Sec. 3.1.1, the basis reproduced
 * exactly by cubic-spline interpolation). */
double oracle_bspline3(double t);

/* Keys' cubic convolution kernel with a = -1/2 (R. G. Keys, "Cubic
 * convolution interpolation for digital image processing", IEEE Trans. ASSP
 * 29, 1981): a cheaper alternative to the cubic spline that interpolates the
 * data directly, with no prefilter.  W(t) = 1 - (5/2)|t|^2 + (3/2)|t|^3 for
 * |t| <= 1, -(1/2)(|t| - 1)(|t| - 2)^2 for 1 < |t| < 2, 0 beyond. */
double oracle_keys(double t);

/* Whole-sample symmetric (mirror) index into [0, N). */
int64_t oracle_mirror(int64_t i, int64_t N);

/* Mean of an FP32 image in FP64 (flat normalisation). */
double oracle_mean_f32(const float* a, int64_t pitch, int W, int H);

/* Calibrates one frame: v[y*W+x] = (raw - bias - dark*t) / (flat / flat_norm). */
void oracle_calibrate(const uint16_t* raw, int64_t raw_pitch, int W, int H,
                      const float* bias, const float* dark, const float* flat,
                      int64_t master_pitch, double t, double flat_norm, double* v);

/* Solves the cubic-spline interpolation system (c[i-1] + 4 c[i] + c[i+1]) / 6
 * = v[i] with mirror boundary conditions along one line of N samples. */
void oracle_spline_solve_line(const double* v, int64_t vstride, double* c, int64_t cstride,
                              int N, double* work /* 2N doubles */);

/* 2-D spline coefficients: the line solve along every row, then every column. */
void oracle_spline_coeffs(const double* v, int W, int H, double* c);

/* Resamples one value at output pixel (x, y) from frame data ``f`` (the
 * calibrated frame for nearest/bilinear, the spline coefficients for spline3).
 * Returns 1 and writes *a if the sample is valid, else returns 0. */
int oracle_sample(const double* f, int W, int H, int x, int y, double dx, double dy,
                  int interp, double* a);

/* Resamples a whole frame.  Invalid outputs get a = 0 and valid = 0. */
void oracle_shift(const double* v, int W, int H, double dx, double dy, int interp,
                  double* a, uint8_t* valid);

/* Sigma-clipped mean of the valid entries of x[0..n).  Writes the mean (NaN if
 * nothing is valid), the kept count, the rejected flags (nullable), the
 * smallest distance of any tested sample to its threshold in units of sigma
 * (+inf if no pass had sigma > 0) and, nullable, the smallest such distance in
 * the data's own units (| |x - centre| - kappa sigma |, over every pass). */
void oracle_clip(const double* x, const uint8_t* valid, int n, const oracle_clip_params* p,
                 double* mean, int* nkept, uint8_t* rejected, double* min_margin,
                 double* min_margin_adu);

/* Median of the valid entries (mean of the two middle values for even counts). */
double oracle_median(const double* x, const uint8_t* valid, int n);

/* Clip + median of every pixel of an aligned stack [n][P] (P pixels). */
void oracle_combine_stack(const double* stack, const uint8_t* valid, int n, int64_t P,
                          const oracle_clip_params* clip, int nthreads, double* mean,
                          double* median, int32_t* nkept, double* min_margin,
                          double* min_margin_adu, uint8_t* rejected);

/* Whole frame set.  raw frame k starts at raw + k*frame_stride (elements).
 * If npix > 0 only the output pixels (px[i], py[i]) are computed and written at
 * index i; else the full W*H grid is written row-major.  stack/valid (nullable,
 * full-grid mode only) receive the aligned samples [n][H][W].
 * nthreads > 1 uses OpenMP.  Returns 0 on success, nonzero on bad input. */
int oracle_reduce_set(const uint16_t* raw, int64_t raw_pitch, int64_t frame_stride,
                      int W, int H, int n,
                      const float* bias, const float* dark, const float* flat,
                      int64_t master_pitch, const double* exptime,
                      const double* dx, const double* dy, int interp, int normalize_flat,
                      const oracle_clip_params* clip, int nthreads,
                      int64_t npix, const int32_t* px, const int32_t* py,
                      double* mean, double* median, int32_t* nkept, double* min_margin,
                      double* min_margin_adu, double* stack, uint8_t* valid);

/* oracle_reduce_set with bad-pixel masking (Sec. 2.1): a source pixel is bad
 * when mask[j*mask_pitch + i] != 0 (mask may be NULL) or its raw value is at
 * least `saturation` (<= 0: off); a sample whose taps with non-zero weight
 * include a bad pixel is invalid and left out of the combine.  frame_norm is
 * an ORACLE_NORM_* mode; returns 2 when a SCALE statistic is 0 or not
 * finite. */
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
                             int frame_norm);

#ifdef __cplusplus
}
#endif
#endif

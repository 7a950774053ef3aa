// combine.cuh -- per-pixel co-adding of an aligned stack held in registers.
//
// Sec. 2.1: the frames are co-added by a sigma-clipped mean; the median is
// produced beside it.  Each thread owns one output pixel and its N samples.
// Invalid samples are +inf, so after an ascending sort the m valid samples
// occupy s[0..m).  Because every clipping pass removes the samples farther
// than kappa*sigma from the centre, the survivors always form one contiguous
// run s[lo..hi) of the sorted samples, so each pass only moves lo and hi.
#pragma once

#include <math.h>
#include <stdint.h>

namespace irp {

struct ClipArgs {
  float kappa_lo, kappa_hi;
  int max_iter, center, ddof;
};

// Batcher's odd-even merge sort on N registers (ascending).  For N not a
// power of two the comparators that would touch an index >= N are dropped,
// which is the network of the next power of two with +inf padding.  The
// comparator list is built at compile time so that one flat, fully unrolled
// loop keeps every index a constant and the samples stay in registers.
template <int N>
struct BatcherNet {
  __host__ __device__ static constexpr int count() {
    int c = 0;
    for (int p = 1; p < N; p <<= 1)
      for (int k = p; k >= 1; k >>= 1)
        for (int j = k % p; j + k < N; j += 2 * k)
          for (int i = 0; i < k; ++i)
            if (i + j + k < N && (i + j) / (2 * p) == (i + j + k) / (2 * p)) ++c;
    return c;
  }
  static constexpr int kCount = count() > 0 ? count() : 1;
  int lo[kCount], hi[kCount];
  __host__ __device__ constexpr BatcherNet() : lo(), hi() {
    int c = 0;
    for (int p = 1; p < N; p <<= 1)
      for (int k = p; k >= 1; k >>= 1)
        for (int j = k % p; j + k < N; j += 2 * k)
          for (int i = 0; i < k; ++i)
            if (i + j + k < N && (i + j) / (2 * p) == (i + j + k) / (2 * p)) {
              lo[c] = i + j;
              hi[c] = i + j + k;
              ++c;
            }
  }
};

template <int N>
__device__ __forceinline__ void sort_network(float (&s)[N]) {
  constexpr BatcherNet<N> net{};
#pragma unroll
  for (int c = 0; c < BatcherNet<N>::count(); ++c) {
    const float a = s[net.lo[c]], b = s[net.hi[c]];
    s[net.lo[c]] = fminf(a, b);
    s[net.hi[c]] = fmaxf(a, b);
  }
}

// s[idx] for a run-time idx without local-memory indexing.
template <int N>
__device__ __forceinline__ float select_at(const float (&s)[N], int idx) {
  float r = s[0];
#pragma unroll
  for (int j = 1; j < N; ++j) r = (j == idx) ? s[j] : r;
  return r;
}

struct CombineOut {
  float mean, median;
  int kept;
  float lo_val, hi_val;  // survivors are the valid samples within [lo_val, hi_val]
};

// s: sorted samples, m valid.  Returns the sigma-clipped mean, the median of
// all valid samples, the survivor count and the survivor value range.
template <int N>
__device__ __forceinline__ CombineOut combine_sorted(const float (&s)[N], int m,
                                                     const ClipArgs& c) {
  CombineOut o;
  if (m <= 0) {
    o.mean = __int_as_float(0x7fffffff);
    o.median = o.mean;
    o.kept = 0;
    o.lo_val = 1.0f;
    o.hi_val = 0.0f;
    return o;
  }
  if (m == N && c.center == 0 && c.max_iter > 0 && N - c.ddof > 0) {
    // All N samples valid (the common case with an exact register bucket): the
    // median and run ends have constant indices, and the first pass needs no
    // range test.  It returns unless the first pass rejects something.
    const float a = s[(N - 1) >> 1], b = s[N >> 1];
    o.median = __fmul_rn(__fadd_rn(a, b), 0.5f);
    const float r = a;
    float S = 0.0f, C = 0.0f, Q = 0.0f;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const float d = __fsub_rn(s[j], r);
      const float y = __fsub_rn(d, C);
      const float t = __fadd_rn(S, y);
      C = __fsub_rn(__fsub_rn(t, S), y);
      S = t;
      Q = __fmaf_rn(d, d, Q);
    }
    const float cd = __fdiv_rn(S, (float)N);
    float ss = __fmaf_rn(cd, __fmaf_rn((float)N, cd, -2.0f * S), Q);
    ss = fmaxf(ss, 0.0f);
    const float sigma = sqrtf(__fdiv_rn(ss, (float)(N - c.ddof)));
    const float elo = __fsub_rn(__fsub_rn(s[0], r), cd);
    const float ehi = __fsub_rn(__fsub_rn(s[N - 1], r), cd);
    if (!(sigma > 0.0f) || (!(-elo > c.kappa_lo * sigma) && !(ehi > c.kappa_hi * sigma))) {
      o.kept = N;
      o.mean = __fadd_rn(r, __fdiv_rn(S, (float)N));
      o.lo_val = s[0];
      o.hi_val = s[N - 1];
      return o;
    }
  }
  const float a = select_at(s, (m - 1) >> 1);
  const float b = select_at(s, m >> 1);
  o.median = __fmul_rn(__fadd_rn(a, b), 0.5f);
  // Reference for shifted sums: a sample at the centre of the run, so that
  // the squared deviations carry no cancellation.
  const float r = a;
  int lo = 0, hi = m;
  // Kahan-compensated sum S (+C) of the deviations over [lo, hi) (a cosmic ray
  // in the first pass must not move the centre); `have` marks S as current.
  float S = 0.0f, C = 0.0f;
  bool have = false;
  for (int it = 0; it < c.max_iter; ++it) {
    const int mm = hi - lo;
    if (mm - c.ddof <= 0) break;
    float Q = 0.0f;
    S = 0.0f;
    C = 0.0f;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const bool in = (unsigned)(j - lo) < (unsigned)mm;
      const float d = in ? __fsub_rn(s[j], r) : 0.0f;
      const float y = __fsub_rn(d, C);
      const float t = __fadd_rn(S, y);
      C = __fsub_rn(__fsub_rn(t, S), y);
      S = t;
      Q = __fmaf_rn(d, d, Q);
    }
    have = true;
    float cd;  // centre - r
    if (c.center == 1) {
      const float qa = select_at(s, lo + ((mm - 1) >> 1));
      const float qb = select_at(s, lo + (mm >> 1));
      cd = __fsub_rn(__fmul_rn(__fadd_rn(qa, qb), 0.5f), r);
    } else {
      cd = __fdiv_rn(S, (float)mm);
    }
    // sum (x - centre)^2 = Q - 2 cd S + mm cd^2
    float ss = __fmaf_rn(cd, __fmaf_rn((float)mm, cd, -2.0f * S), Q);
    ss = fmaxf(ss, 0.0f);
    const float sigma = sqrtf(__fdiv_rn(ss, (float)(mm - c.ddof)));
    if (!(sigma > 0.0f)) break;
    const float tlo = c.kappa_lo * sigma, thi = c.kappa_hi * sigma;
    // survivors are a run of the sorted samples, so the rejected ones are a
    // prefix (below) and a suffix (above) of [lo, hi): when neither extreme
    // is rejected, nothing is
    {
      const float elo = __fsub_rn(__fsub_rn(select_at(s, lo), r), cd);
      const float ehi = __fsub_rn(__fsub_rn(select_at(s, hi - 1), r), cd);
      if (!(-elo > tlo) && !(ehi > thi)) break;
    }
    int nlo = 0, nhi = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const bool in = (unsigned)(j - lo) < (unsigned)mm;
      const float e = __fsub_rn(__fsub_rn(s[j], r), cd);
      nlo += (in & (-e > tlo)) ? 1 : 0;
      nhi += (in & (e > thi)) ? 1 : 0;
    }
    if (nlo + nhi == 0) break;
    lo += nlo;
    hi -= nhi;
    if (hi < lo) hi = lo;
    have = false;
  }
  if (!have) {
    const int mm = hi - lo;
    S = 0.0f;
    C = 0.0f;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const bool in = (unsigned)(j - lo) < (unsigned)mm;
      const float y = __fsub_rn(in ? __fsub_rn(s[j], r) : 0.0f, C);
      const float t = __fadd_rn(S, y);
      C = __fsub_rn(__fsub_rn(t, S), y);
      S = t;
    }
  }
  o.kept = hi - lo;
  o.mean = o.kept > 0 ? __fadd_rn(r, __fdiv_rn(S, (float)o.kept)) : __int_as_float(0x7fffffff);
  o.lo_val = o.kept > 0 ? select_at(s, lo) : 1.0f;
  o.hi_val = o.kept > 0 ? select_at(s, hi - 1) : 0.0f;
  return o;
}

}  // namespace irp

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

// ---------------------------------------------------------------------------
// Clip with a compile-time count M of valid samples (the interior of a set
// whose frame count is M).  The deviations from the lower median are summed
// outward from the median, the lower half downward and the upper half
// upward, so the extreme samples are added last; the running sums are kept
// after each of the K outermost samples of either side.  A pass then needs no
// loop over the samples: the survivors [nlo, M - nhi) have the sums
// SL[nlo] + SU[nhi], and the rejected counts come from the K + 1 outermost
// samples of each side.  The outliers never enter the sums of the survivors,
// so there is no cancellation to compensate.  Returns false (the caller runs
// the general loop) when a side rejects more than K samples.
// ---------------------------------------------------------------------------
constexpr int kClipK = 3;

__host__ __device__ constexpr int clip_min(int a, int b) { return a < b ? a : b; }

template <int N, int M>
__device__ __forceinline__ bool clip_fixed_count(const float (&s)[N], const ClipArgs& c,
                                                 CombineOut& o) {
  static_assert(M >= 3 && M <= N, "fixed-count clip needs 3..N samples");
  constexpr int h = (M + 1) / 2;                    // lower half [0, h), lower median at h - 1
  constexpr int KL = clip_min(kClipK, h - 1);       // partials cover nlo <= KL
  constexpr int KU = clip_min(kClipK, M - h - 1);   // and nhi <= KU
  const float a = s[(M - 1) / 2], b = s[M / 2];
  const float r = a;
  float SL[KL + 1], QL[KL + 1], SU[KU + 1], QU[KU + 1];
  {
    float S = 0.0f, Q = 0.0f;
#pragma unroll
    for (int j = h - 1; j >= 0; --j) {
      const float d = __fsub_rn(s[j], r);
      S = __fadd_rn(S, d);
      Q = __fmaf_rn(d, d, Q);
      if (j <= KL) {
        SL[j] = S;
        QL[j] = Q;
      }
    }
  }
  {
    float S = 0.0f, Q = 0.0f;
#pragma unroll
    for (int j = h; j < M; ++j) {
      const float d = __fsub_rn(s[j], r);
      S = __fadd_rn(S, d);
      Q = __fmaf_rn(d, d, Q);
      if (j >= M - 1 - KU) {
        SU[M - 1 - j] = S;
        QU[M - 1 - j] = Q;
      }
    }
  }
  int nlo = 0, nhi = 0;
#pragma unroll 1
  for (int it = 0; it < c.max_iter; ++it) {
    const int mm = M - nlo - nhi;
    if (mm - c.ddof <= 0) break;
    const float S = __fadd_rn(select_at(SL, nlo), select_at(SU, nhi));
    const float Q = __fadd_rn(select_at(QL, nlo), select_at(QU, nhi));
    const float cd = __fdiv_rn(S, (float)mm);  // centre - r
    // sum (x - centre)^2 = Q - 2 cd S + mm cd^2
    float ss = __fmaf_rn(cd, __fmaf_rn((float)mm, cd, -2.0f * S), Q);
    ss = fmaxf(ss, 0.0f);
    const float sigma = sqrtf(__fdiv_rn(ss, (float)(mm - c.ddof)));
    if (!(sigma > 0.0f)) break;
    const float tlo = c.kappa_lo * sigma, thi = c.kappa_hi * sigma;
    // the rejected samples below (above) the centre are a prefix (suffix) of
    // the sorted run, so counting over all of the outermost samples and
    // keeping the larger count gives the cumulative rejection
    int clo = 0, chi = 0;
#pragma unroll
    for (int j = 0; j <= KL; ++j) clo += (-__fsub_rn(__fsub_rn(s[j], r), cd) > tlo) ? 1 : 0;
#pragma unroll
    for (int k = 0; k <= KU; ++k)
      chi += (__fsub_rn(__fsub_rn(s[M - 1 - k], r), cd) > thi) ? 1 : 0;
    if (clo > KL || chi > KU) return false;
    clo = max(clo, nlo);
    chi = max(chi, nhi);
    if (clo == nlo && chi == nhi) break;
    nlo = clo;
    nhi = chi;
  }
  const int mm = M - nlo - nhi;
  const float S = __fadd_rn(select_at(SL, nlo), select_at(SU, nhi));
  o.median = __fmul_rn(__fadd_rn(a, b), 0.5f);
  o.kept = mm;
  o.mean = __fadd_rn(r, __fdiv_rn(S, (float)mm));
  float lv = s[0], hv = s[M - 1];
#pragma unroll
  for (int j = 1; j <= KL; ++j) lv = (nlo == j) ? s[j] : lv;
#pragma unroll
  for (int k = 1; k <= KU; ++k) hv = (nhi == k) ? s[M - 1 - k] : hv;
  o.lo_val = lv;
  o.hi_val = hv;
  return true;
}

// The register bucket below N (frame counts 4, 5, 6, 8, 10, 12, 16, 24, 32,
// 40, 48, 64): every set reduced with bucket N has more frames than this.
__host__ __device__ constexpr int bucket_below(int N) {
  return N > 48 ? 48 : N > 40 ? 40 : N > 32 ? 32 : N > 24 ? 24 : N > 16 ? 16 : N > 12 ? 12
       : N > 10 ? 10 : N > 8 ? 8 : N > 6 ? 6 : N > 5 ? 5 : N > 4 ? 4 : 0;
}

// Largest gap N - m served by a fixed-count instantiation: the frame counts
// that share register bucket N (up to 8 of them).
template <int N>
__host__ __device__ constexpr int clip_max_gap() {
  return clip_min(7, N - bucket_below(N) - 1);
}

template <int N, int G>
__device__ __forceinline__ bool clip_fixed_dispatch(const float (&s)[N], int m, const ClipArgs& c,
                                                    CombineOut& o) {
  if constexpr (G > clip_max_gap<N>() || N - G < 3) {
    return false;
  } else {
    if (m == N - G) return clip_fixed_count<N, N - G>(s, c, o);
    return clip_fixed_dispatch<N, G + 1>(s, m, c, o);
  }
}

// The same clip for any count m in [N - gap, N] in one code path (for warps
// whose lanes hold different counts, e.g. under a bad-pixel mask, where the
// per-count instantiations would run one after another).  Positions that
// depend on m are picked from short candidate ranges, and the sums add zeros
// at the positions outside this pixel's halves, so every sum, partial and
// decision is the same FP32 sequence as in clip_fixed_count<N, m>.
template <int N>
__device__ __forceinline__ bool clip_window(const float (&s)[N], int m, const ClipArgs& c,
                                            CombineOut& o) {
  constexpr int K = kClipK;
  constexpr int MLO = N - clip_max_gap<N>();  // smallest count handled
  static_assert(MLO >= 9, "window clip needs at least 9 samples (constant K per side)");
  if (m < MLO || m > N) return false;
  constexpr int HLO = (MLO + 1) / 2, HHI = (N + 1) / 2;
  static_assert(HHI <= MLO, "lower halves lie below every count");
  const int h = (m + 1) / 2;
  float a = s[(MLO - 1) / 2], b = s[MLO / 2];
#pragma unroll
  for (int i = (MLO - 1) / 2 + 1; i <= (N - 1) / 2; ++i) a = ((m - 1) / 2 == i) ? s[i] : a;
#pragma unroll
  for (int i = MLO / 2 + 1; i <= N / 2; ++i) b = (m / 2 == i) ? s[i] : b;
  const float r = a;
  float SL[K + 1], QL[K + 1], SU[K + 1], QU[K + 1], U[K + 1];
  {
    float S = 0.0f, Q = 0.0f;
#pragma unroll
    for (int j = HHI - 1; j >= 0; --j) {
      float d = __fsub_rn(s[j], r);
      if (j >= HLO) d = (j < h) ? d : 0.0f;
      S = __fadd_rn(S, d);
      Q = __fmaf_rn(d, d, Q);
      if (j <= K) {
        SL[j] = S;
        QL[j] = Q;
      }
    }
  }
  {
    float S = 0.0f, Q = 0.0f;
#pragma unroll
    for (int k = 0; k <= K; ++k) SU[k] = QU[k] = 0.0f;
#pragma unroll
    for (int j = HLO; j < N; ++j) {
      float d = __fsub_rn(s[j], r);
      const bool in = (j >= HHI || j >= h) && (j < MLO || j < m);
      d = in ? d : 0.0f;
      S = __fadd_rn(S, d);
      Q = __fmaf_rn(d, d, Q);
#pragma unroll
      for (int k = 0; k <= K; ++k) {
        if (j >= MLO - 1 - k && j <= N - 1 - k) {
          const bool at = j == m - 1 - k;
          SU[k] = at ? S : SU[k];
          QU[k] = at ? Q : QU[k];
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k <= K; ++k) {
    float u = s[MLO - 1 - k];
#pragma unroll
    for (int j = MLO - k; j <= N - 1 - k; ++j) u = (j == m - 1 - k) ? s[j] : u;
    U[k] = u;
  }
  int nlo = 0, nhi = 0;
#pragma unroll 1
  for (int it = 0; it < c.max_iter; ++it) {
    const int mm = m - nlo - nhi;
    if (mm - c.ddof <= 0) break;
    const float S = __fadd_rn(select_at(SL, nlo), select_at(SU, nhi));
    const float Q = __fadd_rn(select_at(QL, nlo), select_at(QU, nhi));
    const float cd = __fdiv_rn(S, (float)mm);
    float ss = __fmaf_rn(cd, __fmaf_rn((float)mm, cd, -2.0f * S), Q);
    ss = fmaxf(ss, 0.0f);
    const float sigma = sqrtf(__fdiv_rn(ss, (float)(mm - c.ddof)));
    if (!(sigma > 0.0f)) break;
    const float tlo = c.kappa_lo * sigma, thi = c.kappa_hi * sigma;
    int clo = 0, chi = 0;
#pragma unroll
    for (int j = 0; j <= K; ++j) clo += (-__fsub_rn(__fsub_rn(s[j], r), cd) > tlo) ? 1 : 0;
#pragma unroll
    for (int k = 0; k <= K; ++k) chi += (__fsub_rn(__fsub_rn(U[k], r), cd) > thi) ? 1 : 0;
    if (clo > K || chi > K) return false;
    clo = max(clo, nlo);
    chi = max(chi, nhi);
    if (clo == nlo && chi == nhi) break;
    nlo = clo;
    nhi = chi;
  }
  const int mm = m - nlo - nhi;
  const float S = __fadd_rn(select_at(SL, nlo), select_at(SU, nhi));
  o.median = __fmul_rn(__fadd_rn(a, b), 0.5f);
  o.kept = mm;
  o.mean = __fadd_rn(r, __fdiv_rn(S, (float)mm));
  float lv = s[0];
#pragma unroll
  for (int j = 1; j <= K; ++j) lv = (nlo == j) ? s[j] : lv;
  o.lo_val = lv;
  o.hi_val = select_at(U, nhi);
  return true;
}

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
  if (c.center == 0) {
    if constexpr (N >= 16) {
      // lanes of this warp holding different counts share one code path
      const unsigned act = __activemask();
      if (__match_any_sync(act, m) != act) {
        float t[N];  // a copy for the count-generic path
#pragma unroll
        for (int j = 0; j < N; ++j) t[j] = s[j];
        if (clip_window<N>(t, m, c, o)) return o;
      } else if (clip_fixed_dispatch<N, 0>(s, m, c, o)) {
        return o;
      }
    } else if (clip_fixed_dispatch<N, 0>(s, m, c, o)) {
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

// wide.cuh -- combination (Sec. 2.1 co-adding) of stacks deeper than the
// per-thread register buckets: one warp per output pixel.
//
// The pixel's samples are spread over the 32 lanes in lane-major blocks of J
// (sample e = lane * J + i in register i), sorted by a bitonic network whose
// short strides run inside a lane and whose long strides pair lanes through
// shuffles.  The clip then works as in the register path: survivors are a
// run [lo, hi) of the sorted samples, each pass sums the deviations from the
// lower median over the run (Kahan-compensated per lane, double-float across
// the lanes) and counts the rejected prefix and suffix.  Every reduction is a
// butterfly, so all lanes hold the same values and take the same branches.
#pragma once

#include "combine.cuh"
#include "common.cuh"

namespace irp {

constexpr int kWideThreads = 256;  // 8 warps, 32 pixels of one output row per CTA
constexpr int kWideMaxFrames = IRP_MAX_WIDE_FRAMES;

// Samples per lane for n frames: the sort length 32 J is a power of two >= n.
__host__ __device__ constexpr int wide_j(int n) {
  return n <= 128 ? 4 : (n <= 256 ? 8 : (n <= 512 ? 16 : 32));
}

// Shared-memory position of sample e of pixel p.  A pixel's samples are
// contiguous with one pad word after every J of them, and the pixel stride is
// odd, so the staging stores (one frame, 32 pixels) and the sort's loads (one
// pixel, lane-major blocks of J) each touch 32 distinct banks.
template <int J>
struct WideSmem {
  static constexpr int kPixStride = 32 * (J + 1) + 1;  // 32 blocks of J + pad, odd
  static constexpr size_t kBytes = (size_t)32 * kPixStride * sizeof(float);
  __device__ static __forceinline__ int at(int p, int e) { return p * kPixStride + e + e / J; }
};

// Ascending bitonic sort of the warp's 32 J values (lane-major blocks), in
// the form whose merges start with a mirrored compare (element e against
// e ^ (s - 1)) and continue with ascending half-cleaners: every compare keeps
// the minimum at the lower index, so the in-lane ones need no direction test.
template <int J>
__device__ __forceinline__ void warp_bitonic_sort(float (&v)[J], int lane) {
  constexpr int L = 32 * J;
#pragma unroll
  for (int s = 2; s <= L; s <<= 1) {
    if (s <= J) {
      // mirrored compare inside the lane: i against i ^ (s - 1)
#pragma unroll
      for (int i = 0; i < J; ++i) {
        if (i & (s >> 1)) continue;
        const int j = i ^ (s - 1);
        const float a = v[i], b = v[j];
        v[i] = fminf(a, b);
        v[j] = fmaxf(a, b);
      }
    } else {
      // mirrored compare across lanes: (lane, i) against (lane ^ (s/J - 1), J-1-i)
      const int lm = s / J - 1;
      const bool lower = (lane & ((s >> 1) / J)) == 0;
      float p[J];
#pragma unroll
      for (int i = 0; i < J; ++i) p[i] = __shfl_xor_sync(0xffffffffu, v[J - 1 - i], lm);
#pragma unroll
      for (int i = 0; i < J; ++i) v[i] = lower ? fminf(v[i], p[i]) : fmaxf(v[i], p[i]);
    }
#pragma unroll
    for (int d = s >> 2; d > 0; d >>= 1) {
      if (d >= J) {
        const int ld = d / J;
        const bool lower = (lane & ld) == 0;
#pragma unroll
        for (int i = 0; i < J; ++i) {
          const float p = __shfl_xor_sync(0xffffffffu, v[i], ld);
          v[i] = lower ? fminf(v[i], p) : fmaxf(v[i], p);
        }
      } else {
#pragma unroll
        for (int i = 0; i < J; ++i) {
          if (i & d) continue;
          const float a = v[i], b = v[i ^ d];
          v[i] = fminf(a, b);
          v[i ^ d] = fmaxf(a, b);
        }
      }
    }
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum over the warp of the double-float values (hi, lo), rounded to FP32.
__device__ __forceinline__ float warp_sum_df(float hi, float lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float bh = __shfl_xor_sync(0xffffffffu, hi, o);
    const float bl = __shfl_xor_sync(0xffffffffu, lo, o);
    // two-sum of the high parts (Knuth), then the low parts and renormalise
    const float s = __fadd_rn(hi, bh);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
    const float t = __fadd_rn(e, __fadd_rn(lo, bl));
    hi = __fadd_rn(s, t);
    lo = __fsub_rn(t, __fsub_rn(hi, s));
  }
  return __fadd_rn(hi, lo);
}

struct WideOut {
  float mean, median, lo_val, hi_val;
  int kept;
};

// Kahan-compensated sum over the warp of the deviations dv[e] for e in
// [lo, lo + mm), and (optionally) the plain sum of their squares.
template <int J, bool SQ>
__device__ __forceinline__ float wide_run_sums(const float (&dv)[J], int lane, int lo, int mm,
                                               float* q_out) {
  float S = 0.0f, C = 0.0f, Q = 0.0f;
#pragma unroll
  for (int i = 0; i < J; ++i) {
    const bool in = (unsigned)(lane * J + i - lo) < (unsigned)mm;
    const float d = in ? dv[i] : 0.0f;
    const float y = __fsub_rn(d, C);
    const float t = __fadd_rn(S, y);
    C = __fsub_rn(__fsub_rn(t, S), y);
    S = t;
    if (SQ) Q = __fmaf_rn(d, d, Q);
  }
  if (SQ) *q_out = warp_sum(Q);
  return warp_sum_df(S, -C);
}

// Sigma-clipped mean (cumulative rejection, at most max_iter passes) and
// median of the m valid samples, sorted to the front of v.  `run` holds the
// same sorted values in shared memory (sample e at run[e + e / J]), from which
// the order statistics are read.
template <int J>
__device__ __forceinline__ WideOut wide_combine(const float (&v)[J], const float* run, int m,
                                                const ClipArgs& c, int lane) {
  WideOut o;
  const float kNaN = __int_as_float(0x7fffffff);
  auto at = [&](int e) { return run[e + e / J]; };
  if (m <= 0) {
    o.mean = kNaN;
    o.median = kNaN;
    o.kept = 0;
    o.lo_val = 1.0f;
    o.hi_val = 0.0f;
    return o;
  }
  const float a = at((m - 1) >> 1);
  const float b = at(m >> 1);
  o.median = __fmul_rn(__fadd_rn(a, b), 0.5f);
  const float r = a;  // reference of the shifted sums: no cancellation in the squares
  float dv[J];        // deviations from r (+inf for invalid samples)
#pragma unroll
  for (int i = 0; i < J; ++i) dv[i] = __fsub_rn(v[i], r);
  int lo = 0, hi = m;
  float S = 0.0f;
  bool have = false;
  for (int it = 0; it < c.max_iter; ++it) {
    const int mm = hi - lo;
    if (mm - c.ddof <= 0) break;
    float Q;
    S = wide_run_sums<J, true>(dv, lane, lo, mm, &Q);
    have = true;
    float cd;  // centre - r
    if (c.center == 1) {
      const float qa = at(lo + ((mm - 1) >> 1));
      const float qb = at(lo + (mm >> 1));
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
    // the rejected samples are a prefix and a suffix of the run
    const bool rlo = -__fsub_rn(__fsub_rn(at(lo), r), cd) > tlo;
    const bool rhi = __fsub_rn(__fsub_rn(at(hi - 1), r), cd) > thi;
    if (!rlo && !rhi) break;
    // Both tests are monotone in the sample value and the run is sorted: when
    // the run's lowest sample is rejected, so is every sample below the run,
    // and no sample above it; likewise at the top, where the invalid samples
    // (+inf) and those already rejected all pass the test.
    int clo = 0, chi = 0;
#pragma unroll
    for (int i = 0; i < J; ++i) {
      const float d = __fsub_rn(dv[i], cd);
      clo += (-d > tlo) ? 1 : 0;
      chi += (d > thi) ? 1 : 0;
    }
    const int nlo = rlo ? min(__reduce_add_sync(0xffffffffu, clo) - lo, mm) : 0;
    const int nhi = rhi ? min(__reduce_add_sync(0xffffffffu, chi) - (32 * J - hi), mm - nlo) : 0;
    lo += nlo;
    hi -= nhi;
    have = false;
  }
  if (!have) S = wide_run_sums<J, false>(dv, lane, lo, hi - lo, nullptr);
  o.kept = hi - lo;
  o.mean = o.kept > 0 ? __fadd_rn(r, __fdiv_rn(S, (float)o.kept)) : kNaN;
  o.lo_val = o.kept > 0 ? at(lo) : 1.0f;
  o.hi_val = o.kept > 0 ? at(hi - 1) : 0.0f;
  return o;
}

}  // namespace irp

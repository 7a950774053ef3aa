// wide.cuh -- combination (Sec. 2.1 co-adding) of stacks deeper than the
// per-thread register buckets: a group of G lanes per output pixel.
//
// A pixel's samples are spread over its group's G lanes in lane-major blocks
// of J (sample e = t * J + i in register i of the group's lane t), and sorted
// by a bitonic network whose short strides run inside a lane and whose long
// strides pair lanes of the group through shuffles.  The clip then works as
// in the register path: survivors are a run [lo, hi) of the sorted samples,
// each pass sums the deviations from the lower median over the run
// (Kahan-compensated per lane, double-float across the group) and counts the
// rejected prefix and suffix.  Every reduction is a butterfly inside the
// group, so the group's lanes hold the same values; the warp's groups run the
// clip passes in lockstep until none of them continues.
#pragma once

#include "combine.cuh"
#include "common.cuh"

namespace irp {

constexpr int kWideThreads = 256;  // 8 warps, 32 pixels of one output row per CTA
constexpr int kWideMaxFrames = IRP_MAX_WIDE_FRAMES;

// Lanes per pixel (G) and samples per lane (J) for n frames: the sort length
// G J is the power of two >= n, with 32 samples per lane, so that only the
// sort stages of stride 32 or more cross lanes.
__host__ __device__ constexpr int wide_g(int n) {
  return n <= 128 ? 4 : (n <= 256 ? 8 : (n <= 512 ? 16 : 32));
}
__host__ __device__ constexpr int wide_j(int n) { return 32; }

// Shared-memory position of sample e of pixel p.  A pixel's samples are
// contiguous with one pad word after every J of them, and the pixel stride
// G (J + 1) + 1 is odd.  The staging stores (one frame, 32 pixels) then
// touch 32 distinct banks, and so do the sort's loads, where the warp's
// 32 / G groups read pixels 32 / (32 / G) apart in lane-major blocks of J.
template <int G, int J>
struct WideSmem {
  static constexpr int kPixStride = G * (J + 1) + 1;
  static constexpr size_t kBytes = (size_t)32 * kPixStride * sizeof(float);
  __device__ static __forceinline__ int at(int p, int e) { return p * kPixStride + e + e / J; }
};

// Ascending bitonic sort of the group's G J values (lane-major blocks; t is
// the lane's index in its group), in the form whose merges start with a
// mirrored compare (element e against e ^ (s - 1)) and continue with
// ascending half-cleaners: every compare keeps the minimum at the lower
// index, so the in-lane ones need no direction test.  Cross-lane partners
// differ in lane bits below G, so a shuffle never leaves the group.
template <int G, int J>
__device__ __forceinline__ void group_bitonic_sort(float (&v)[J], int t) {
  constexpr int L = G * J;
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
      // mirrored compare across lanes: (t, i) against (t ^ (s/J - 1), J-1-i)
      const int lm = s / J - 1;
      const bool lower = (t & ((s >> 1) / J)) == 0;
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
        const bool lower = (t & ld) == 0;
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

template <int G>
__device__ __forceinline__ int group_sum_i(int v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum over the group of the double-float values (hi, lo), rounded to FP32.
template <int G>
__device__ __forceinline__ float group_sum_df(float hi, float lo) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
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

// Kahan-compensated sum over the group of the deviations dv[e] for e in
// [lo, lo + mm), and (optionally) the plain sum of their squares.
template <int G, int J, bool SQ>
__device__ __forceinline__ float group_run_sums(const float (&dv)[J], int t, int lo, int mm,
                                                float* q_out) {
  float S = 0.0f, C = 0.0f, Q = 0.0f;
#pragma unroll
  for (int i = 0; i < J; ++i) {
    const bool in = (unsigned)(t * J + i - lo) < (unsigned)mm;
    const float d = in ? dv[i] : 0.0f;
    const float y = __fsub_rn(d, C);
    const float s = __fadd_rn(S, y);
    C = __fsub_rn(__fsub_rn(s, S), y);
    S = s;
    if (SQ) Q = __fmaf_rn(d, d, Q);
  }
  if (SQ) *q_out = group_sum<G>(Q);
  return group_sum_df<G>(S, -C);
}

// Sigma-clipped mean (cumulative rejection, at most max_iter passes) and
// median of the m valid samples of the group's pixel, sorted to the front of
// v.  `run` holds the same sorted values in shared memory (sample e at
// run[e + e / J]), from which the order statistics are read.  All lanes of
// the warp call this together: a group that has finished keeps its results
// while the others run their next pass, and every shared-memory index stays
// inside the pixel's block.
template <int G, int J>
__device__ __forceinline__ WideOut group_combine(const float (&v)[J], const float* run, int m,
                                                 const ClipArgs& c, int t) {
  constexpr int L = G * J;
  const float kNaN = __int_as_float(0x7fffffff);
  auto at = [&](int e) {
    e = min(max(e, 0), L - 1);
    return run[e + e / J];
  };
  WideOut o;
  const int mi = max(m, 1);
  const float a = at((mi - 1) >> 1);
  const float b = at(mi >> 1);
  o.median = m > 0 ? __fmul_rn(__fadd_rn(a, b), 0.5f) : kNaN;
  const float r = a;  // reference of the shifted sums: no cancellation in the squares
  float dv[J];        // deviations from r (+inf for invalid samples)
#pragma unroll
  for (int i = 0; i < J; ++i) dv[i] = __fsub_rn(v[i], r);
  int lo = 0, hi = m;
  float S = 0.0f;
  bool have = false;
  bool done = m <= 0;
  for (int it = 0; it < c.max_iter; ++it) {
    if (!__any_sync(0xffffffffu, !done)) break;
    const int mm = hi - lo;
    const bool act = !done && mm - c.ddof > 0;
    done = !act;  // a run too short to clip ends the passes
    float Q;
    const float Sp = group_run_sums<G, J, true>(dv, t, lo, mm, &Q);
    if (act) {
      S = Sp;
      have = true;
    }
    const int mq = max(mm, 1);
    float cd;  // centre - r
    if (c.center == 1) {
      const float qa = at(lo + ((mq - 1) >> 1));
      const float qb = at(lo + (mq >> 1));
      cd = __fsub_rn(__fmul_rn(__fadd_rn(qa, qb), 0.5f), r);
    } else {
      cd = __fdiv_rn(Sp, (float)mq);
    }
    // sum (x - centre)^2 = Q - 2 cd S + mm cd^2
    float ss = __fmaf_rn(cd, __fmaf_rn((float)mm, cd, -2.0f * Sp), Q);
    ss = fmaxf(ss, 0.0f);
    const float sigma = sqrtf(__fdiv_rn(ss, (float)max(mm - c.ddof, 1)));
    const bool clip = act && sigma > 0.0f;
    const float tlo = c.kappa_lo * sigma, thi = c.kappa_hi * sigma;
    // the rejected samples are a prefix and a suffix of the run
    const bool rlo = clip && -__fsub_rn(__fsub_rn(at(lo), r), cd) > tlo;
    const bool rhi = clip && __fsub_rn(__fsub_rn(at(hi - 1), r), cd) > thi;
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
    clo = group_sum_i<G>(clo);
    chi = group_sum_i<G>(chi);
    if (rlo || rhi) {
      const int nlo = rlo ? min(clo - lo, mm) : 0;
      const int nhi = rhi ? min(chi - (L - hi), mm - nlo) : 0;
      lo += nlo;
      hi -= nhi;
      have = false;
      done = false;
    } else {
      done = true;  // nothing rejected (or sigma 0): the clip has converged
    }
  }
  if (__any_sync(0xffffffffu, !have && m > 0)) {
    const float Sf = group_run_sums<G, J, false>(dv, t, lo, hi - lo, nullptr);
    if (!have) S = Sf;
  }
  o.kept = m > 0 ? hi - lo : 0;
  o.mean = o.kept > 0 ? __fadd_rn(r, __fdiv_rn(S, (float)o.kept)) : kNaN;
  o.lo_val = o.kept > 0 ? at(lo) : 1.0f;
  o.hi_val = o.kept > 0 ? at(hi - 1) : 0.0f;
  return o;
}

}  // namespace irp

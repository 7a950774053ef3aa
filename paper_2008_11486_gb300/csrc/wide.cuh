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

// Ascending bitonic sort of the warp's 32 J values (lane-major blocks).
template <int J>
__device__ __forceinline__ void warp_bitonic_sort(float (&v)[J], int lane) {
  constexpr int L = 32 * J;
#pragma unroll
  for (int s = 2; s <= L; s <<= 1) {
#pragma unroll
    for (int d = s >> 1; d > 0; d >>= 1) {
      if (d >= J) {
        // partner: the same register of lane ^ (d / J); the lower element of
        // the pair keeps the minimum when its run of length s ascends
        const int ld = d / J;
        const bool asc = ((lane * J) & s) == 0;
        const bool keep_min = asc != ((lane & ld) != 0);
#pragma unroll
        for (int i = 0; i < J; ++i) {
          const float p = __shfl_xor_sync(0xffffffffu, v[i], ld);
          v[i] = keep_min ? fminf(v[i], p) : fmaxf(v[i], p);
        }
      } else {
#pragma unroll
        for (int i = 0; i < J; ++i) {
          if (i & d) continue;
          // runs shorter than a block: direction fixed by i; longer: by the lane
          const bool asc = s < J ? (i & s) == 0 : ((lane * J) & s) == 0;
          const float a = v[i], b = v[i ^ d];
          const float lo = fminf(a, b), hi = fmaxf(a, b);
          v[i] = asc ? lo : hi;
          v[i ^ d] = asc ? hi : lo;
        }
      }
    }
  }
}

// Sorted sample e (warp-uniform e).
template <int J>
__device__ __forceinline__ float wide_at(const float (&v)[J], int e) {
  const int r = e % J;
  float sel = v[0];
#pragma unroll
  for (int i = 1; i < J; ++i) sel = (i == r) ? v[i] : sel;
  return __shfl_sync(0xffffffffu, sel, e / J);
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

// Kahan-compensated sum over the warp of (v[e] - r) for e in [lo, lo + mm),
// and (optionally) the plain sum of their squares.
template <int J, bool SQ>
__device__ __forceinline__ float wide_run_sums(const float (&v)[J], int lane, int lo, int mm,
                                               float r, float* q_out) {
  float S = 0.0f, C = 0.0f, Q = 0.0f;
#pragma unroll
  for (int i = 0; i < J; ++i) {
    const int e = lane * J + i;
    const bool in = (unsigned)(e - lo) < (unsigned)mm;
    const float d = in ? __fsub_rn(v[i], r) : 0.0f;
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
// median of the m valid samples, sorted to the front of v.
template <int J>
__device__ __forceinline__ WideOut wide_combine(const float (&v)[J], int m, const ClipArgs& c,
                                                int lane) {
  WideOut o;
  const float kNaN = __int_as_float(0x7fffffff);
  if (m <= 0) {
    o.mean = kNaN;
    o.median = kNaN;
    o.kept = 0;
    o.lo_val = 1.0f;
    o.hi_val = 0.0f;
    return o;
  }
  const float a = wide_at<J>(v, (m - 1) >> 1);
  const float b = wide_at<J>(v, m >> 1);
  o.median = __fmul_rn(__fadd_rn(a, b), 0.5f);
  const float r = a;  // reference of the shifted sums: no cancellation in the squares
  int lo = 0, hi = m;
  float S = 0.0f;
  bool have = false;
  for (int it = 0; it < c.max_iter; ++it) {
    const int mm = hi - lo;
    if (mm - c.ddof <= 0) break;
    float Q;
    S = wide_run_sums<J, true>(v, lane, lo, mm, r, &Q);
    have = true;
    float cd;  // centre - r
    if (c.center == 1) {
      const float qa = wide_at<J>(v, lo + ((mm - 1) >> 1));
      const float qb = wide_at<J>(v, lo + (mm >> 1));
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
    const float elo = __fsub_rn(__fsub_rn(wide_at<J>(v, lo), r), cd);
    const float ehi = __fsub_rn(__fsub_rn(wide_at<J>(v, hi - 1), r), cd);
    if (!(-elo > tlo) && !(ehi > thi)) break;
    int nlo = 0, nhi = 0;
#pragma unroll
    for (int i = 0; i < J; ++i) {
      const int e = lane * J + i;
      const bool in = (unsigned)(e - lo) < (unsigned)mm;
      const float d = __fsub_rn(__fsub_rn(v[i], r), cd);
      nlo += (in & (-d > tlo)) ? 1 : 0;
      nhi += (in & (d > thi)) ? 1 : 0;
    }
    nlo = __reduce_add_sync(0xffffffffu, nlo);
    nhi = __reduce_add_sync(0xffffffffu, nhi);
    if (nlo + nhi == 0) break;
    lo += nlo;
    hi -= nhi;
    if (hi < lo) hi = lo;
    have = false;
  }
  if (!have) S = wide_run_sums<J, false>(v, lane, lo, hi - lo, r, nullptr);
  o.kept = hi - lo;
  o.mean = o.kept > 0 ? __fadd_rn(r, __fdiv_rn(S, (float)o.kept)) : kNaN;
  o.lo_val = o.kept > 0 ? wide_at<J>(v, lo) : 1.0f;
  o.hi_val = o.kept > 0 ? wide_at<J>(v, hi - 1) : 0.0f;
  return o;
}

}  // namespace irp

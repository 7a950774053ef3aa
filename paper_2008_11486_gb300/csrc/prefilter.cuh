// prefilter.cuh -- cubic-spline coefficients of calibrated frames.
#pragma once

#include "reduce_tile.cuh"

namespace irp {

// ---------------------------------------------------------------------------
// Cubic-spline prefilter of calibrated raw frames (Sec. 3.2.1: one tridiagonal
// system per row and per column).  The exact solution of the mirror-boundary
// system equals the convolution of the mirror-extended data with
// h[k] = sqrt(3) z1^|k|, z1 = sqrt(3) - 2, which splits into a causal and an
// anti-causal first-order recursion: c = sqrt(3) (y+ + y- - v).  Each CTA
// computes the coefficients of a kPrefTile^2 tile of one frame from a window
// with kPrefHalo samples of recursion warm-up on every side; positions outside
// the frame read the mirror-extended data, so the frame edges are exact.
// Rows first, then columns (the 2-D system is separable).
// ---------------------------------------------------------------------------
template <int SRC>
__device__ __forceinline__ float pref_load(const SetDesc& S, const FrameDesc& F, int gx, int gy,
                                           float flat_norm, uint32_t* status) {
  if (SRC == SRC_RAW) {
    const int64_t m = (int64_t)gy * S.master_pitch + gx;
    const uint16_t q = __ldg((const uint16_t*)F.src + (int64_t)gy * S.src_pitch + gx);
    const float rf = inv_flat(__ldg(S.flat + m), flat_norm, status);
    return calibrate_px(q, __ldg(S.bias + m), __ldg(S.dark + m), F.t, rf);
  } else if (SRC == SRC_F32) {
    return __ldg((const float*)F.src + (int64_t)gy * S.src_pitch + gx);
  } else {
    const __half q = ((const __half*)F.src)[(int64_t)gy * S.src_pitch + gx];
    return __half2float(q);  // spline of h; scale/offset are applied by the caller
  }
}

constexpr int kPrefWS = kPrefWin + 1;   // row stride of the window (bank spread)
constexpr int kPrefTS = kPrefTile + 1;  // row stride of the partial-result arrays

inline size_t prefilter_smem_bytes() {
  return sizeof(float) * ((size_t)kPrefWin * kPrefWS + 2 * (size_t)kPrefWin * kPrefTS);
}

template <int SRC>
__global__ void __launch_bounds__(kThreads)
    k_prefilter(const __grid_constant__ InlinePlan inl, const void* plan_dev) {
  extern __shared__ float4 smem4[];
  float* v = reinterpret_cast<float*>(smem4);  // [kPrefWin][kPrefWS]
  float* A = v + kPrefWin * kPrefWS;            // [kPrefWin][kPrefTS]
  float* B = A + kPrefWin * kPrefTS;            // [kPrefWin][kPrefTS]
  const PlanView P = make_view(inl, plan_dev);
  const int item = blockIdx.x;
  if (item >= P.h->npitems) return;
  // locate the set by its first prefilter item
  int si = 0;
  {
    int lo = 0, hi = P.h->nsets - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (P.sets[mid].ptile0 <= item) lo = mid; else hi = mid - 1;
    }
    si = lo;
  }
  const SetDesc& S = P.sets[si];
  const int per_frame = S.ptiles_x * S.ptiles_y;
  const int local = item - S.ptile0;
  const int k = local / per_frame;
  const int pt = local - k * per_frame;
  const FrameDesc& F = P.frames[S.frame0 + k];
  const int x0 = (pt % S.ptiles_x) * kPrefTile, y0 = (pt / S.ptiles_x) * kPrefTile;
  const int W = S.W, H = S.H;
  float flat_norm = 1.0f;
  if (SRC == SRC_RAW && S.flat_sum) flat_norm = (float)(*S.flat_sum / ((double)W * H));
  uint32_t* status = P.h->status;

  // 1. calibrated, mirror-extended window
  for (int e = threadIdx.x; e < kPrefWin * kPrefWin; e += kThreads) {
    const int r = e / kPrefWin, c = e - r * kPrefWin;
    const int gx = mirror_index(x0 - kPrefHalo + c, W);
    const int gy = mirror_index(y0 - kPrefHalo + r, H);
    v[r * kPrefWS + c] = pref_load<SRC>(S, F, gx, gy, flat_norm, status);
  }
  __syncthreads();
  // 2. row recursions: threads [0, W) causal, [W, 2W) anti-causal (W = window rows)
  const int tid = threadIdx.x;
  if (tid < kPrefWin) {
    const float* row = v + tid * kPrefWS;
    float y = 0.0f;
#pragma unroll 4
    for (int c = 0; c < kPrefHalo + kPrefTile; ++c) {
      y = __fmaf_rn(kZ1, y, row[c]);
      if (c >= kPrefHalo) A[tid * kPrefTS + c - kPrefHalo] = y;
    }
  } else if (tid < 2 * kPrefWin) {
    const int r = tid - kPrefWin;
    const float* row = v + r * kPrefWS;
    float y = 0.0f;
#pragma unroll 4
    for (int c = kPrefWin - 1; c >= kPrefHalo; --c) {
      y = __fmaf_rn(kZ1, y, row[c]);
      if (c < kPrefHalo + kPrefTile) B[r * kPrefTS + c - kPrefHalo] = y;
    }
  }
  __syncthreads();
  // row coefficients of the tile's columns for every window row -> A
  for (int e = tid; e < kPrefWin * kPrefTile; e += kThreads) {
    const int r = e / kPrefTile, c = e - r * kPrefTile;
    const float s = __fsub_rn(__fadd_rn(A[r * kPrefTS + c], B[r * kPrefTS + c]),
                              v[r * kPrefWS + c + kPrefHalo]);
    A[r * kPrefTS + c] = __fmul_rn(kSqrt3, s);
  }
  __syncthreads();
  // 3. column recursions on A: causal -> B, anti-causal -> v (reused)
  if (tid < kPrefTile) {
    float y = 0.0f;
#pragma unroll 4
    for (int r = 0; r < kPrefHalo + kPrefTile; ++r) {
      y = __fmaf_rn(kZ1, y, A[r * kPrefTS + tid]);
      if (r >= kPrefHalo) B[r * kPrefTS + tid] = y;
    }
  } else if (tid < 2 * kPrefTile) {
    const int c = tid - kPrefTile;
    float y = 0.0f;
#pragma unroll 4
    for (int r = kPrefWin - 1; r >= kPrefHalo; --r) {
      y = __fmaf_rn(kZ1, y, A[r * kPrefTS + c]);
      if (r < kPrefHalo + kPrefTile) v[r * kPrefWS + c] = y;
    }
  }
  __syncthreads();
  // 4. c = sqrt(3) (y+ + y- - crow) on the tile, stored densely (pitch W)
  float* out = F.coef;
  for (int e = tid; e < kPrefTile * kPrefTile; e += kThreads) {
    const int r = e / kPrefTile, c = e - r * kPrefTile;
    const int gx = x0 + c, gy = y0 + r;
    if (gx < W && gy < H) {
      const int rr = r + kPrefHalo;
      const float s = __fsub_rn(__fadd_rn(B[rr * kPrefTS + c], v[rr * kPrefWS + c]),
                                A[rr * kPrefTS + c]);
      out[(int64_t)gy * W + gx] = __fmul_rn(kSqrt3, s);
    }
  }
}

}  // namespace irp

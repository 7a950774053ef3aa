// prefilter.cuh -- cubic-spline coefficients of calibrated frames.
//
// Sec. 3.2.1: cubic-spline interpolation solves one tridiagonal system per
// row and per column, (c[i-1] + 4 c[i] + c[i+1]) / 6 = v[i].  With mirror
// boundaries its exact solution is the convolution of the mirror-extended data
// with h[k] = sqrt(3) z1^|k|, z1 = sqrt(3) - 2, i.e. c = sqrt(3)(y+ + y- - v)
// with the causal recursion y+[i] = v[i] + z1 y+[i-1] and the anti-causal one
// y-[i] = v[i] + z1 y-[i+1].  Both are run over independent segments that start
// kPrefHalo samples early (|z1|^17 < 2e-10), so every thread owns a short,
// fully unrolled recursion held in registers.  Positions outside the frame
// read the mirror-extended data, which makes the frame edges exact.
//
// A CTA owns a kPrefTile^2 tile of coefficients and a group of frames of one
// set: the tile's masters are staged in shared memory once and reused by the
// group's frames (raw source).  The coefficients are written to frames padded
// by 2 mirrored samples on every side, pitch S.coef_pitch (multiple of 4), so
// that the resampling kernel reads taps i0-1 .. i0+2 without mirroring.
#pragma once

#include "reduce_tile.cuh"

namespace irp {

constexpr int kPrefExt = kPrefTile + 4;               // coefficients computed per axis
constexpr int kPrefW = kPrefExt + 2 * kPrefHalo;       // window per axis (100)
constexpr int kPrefWS = kPrefW + 1;                    // window row stride
constexpr int kPrefRS = kPrefExt + 1;                  // row-pass result stride
constexpr int kPrefThreads = 288;
constexpr int kPrefRowSeg = kPrefExt / 2;              // 34 outputs per row task
constexpr int kPrefColSeg = kPrefExt / 4;              // 17 outputs per column task
constexpr int kPrefPerThread = (kPrefW * kPrefW + kPrefThreads - 1) / kPrefThreads;  // 35
static_assert(kPrefW * 2 <= kPrefThreads && kPrefExt * 4 <= kPrefThreads, "prefilter tasks");

inline size_t prefilter_smem_bytes(int src) {
  size_t f = (size_t)kPrefW * kPrefWS + (size_t)kPrefW * kPrefRS;
  if (src == SRC_RAW) f += 3 * (size_t)kPrefW * kPrefWS;
  return f * sizeof(float);
}

template <int SRC>
__global__ void __launch_bounds__(kPrefThreads, 1)
    k_prefilter(const __grid_constant__ InlinePlan inl, const void* plan_dev) {
  extern __shared__ float4 smem4[];
  float* v = reinterpret_cast<float*>(smem4);   // [kPrefW][kPrefWS]
  float* R = v + kPrefW * kPrefWS;              // [kPrefW][kPrefRS]
  float* mb = R + kPrefW * kPrefRS;             // masters (raw source)
  float* md = mb + kPrefW * kPrefWS;
  float* mr = md + kPrefW * kPrefWS;
  const PlanView P = make_view(inl, plan_dev);
  const int item = blockIdx.x;
  if (item >= P.h->npitems) return;
  int si = 0;
  {
    int lo = 0, hi = P.h->nsets - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (P.sets[mid].ptile0 <= item) lo = mid; else hi = mid - 1;
    }
    si = lo;
  }
  const SetDesc& S = P.sets[si];
  if (SRC == SRC_RAW && S.ready_flag) {  // the set's raw frames may still be arriving
    __shared__ int s_ok;
    if (threadIdx.x == 0)
      s_ok = wait_ready(S.ready_flag, S.ready_value, P.h->spin_limit, P.h->status);
    __syncthreads();
    if (!s_ok) return;  // status latched
  }
  const int ntiles = S.ptiles_x * S.ptiles_y;
  const int local = item - S.ptile0;
  const int grp = local / ntiles;
  const int pt = local - grp * ntiles;
  const int fpg = S.pframes;  // frames per group
  const int k0 = grp * fpg, k1 = min(S.n, k0 + fpg);
  const int tx = pt % S.ptiles_x, ty = pt / S.ptiles_x;
  const int x0 = tx * kPrefTile, y0 = ty * kPrefTile;
  const int W = S.W, H = S.H;
  const int wx0 = x0 - 2 - kPrefHalo, wy0 = y0 - 2 - kPrefHalo;  // window origin
  const int tid = threadIdx.x;
  uint32_t* status = P.h->status;

  // window element offsets (frame-independent), mirrored at the frame edges
  int goff[kPrefPerThread];
#pragma unroll
  for (int i = 0; i < kPrefPerThread; ++i) {
    const int e = tid + i * kPrefThreads;
    const int r = e / kPrefW, c = e - r * kPrefW;
    const int gx = mirror_index(wx0 + c, W), gy = mirror_index(wy0 + r, H);
    goff[i] = (e < kPrefW * kPrefW) ? gy * (int)S.src_pitch + gx : 0;
  }
  if (SRC == SRC_RAW) {
    const float flat_norm = S.flat_sum ? (float)(*S.flat_sum / ((double)W * H)) : 1.0f;
    for (int e = tid; e < kPrefW * kPrefW; e += kPrefThreads) {
      const int r = e / kPrefW, c = e - r * kPrefW;
      const int gx = mirror_index(wx0 + c, W), gy = mirror_index(wy0 + r, H);
      const int64_t o = (int64_t)gy * S.master_pitch + gx;
      mb[r * kPrefWS + c] = __ldg(S.bias + o);
      md[r * kPrefWS + c] = __ldg(S.dark + o);
      mr[r * kPrefWS + c] = inv_flat(__ldg(S.flat + o), flat_norm, status);
    }
  }
  // owned output range (the padded border belongs to the edge tiles)
  const int ox0 = x0 - (x0 == 0 ? 2 : 0), ox1 = min(x0 + kPrefTile, W) + (x0 + kPrefTile >= W ? 2 : 0);
  const int oy0 = y0 - (y0 == 0 ? 2 : 0), oy1 = min(y0 + kPrefTile, H) + (y0 + kPrefTile >= H ? 2 : 0);

  for (int k = k0; k < k1; ++k) {
    const FrameDesc& F = P.frames[S.frame0 + k];
    __syncthreads();  // previous frame's passes are done with v and R
    // 1. the frame's calibrated, mirror-extended window
#pragma unroll
    for (int i = 0; i < kPrefPerThread; ++i) {
      const int e = tid + i * kPrefThreads;
      if (e < kPrefW * kPrefW) {
        const int r = e / kPrefW, c = e - r * kPrefW;
        const int si_ = r * kPrefWS + c;
        float val;
        if (SRC == SRC_RAW) {
          const uint16_t q = __ldg((const uint16_t*)F.src + goff[i]);
          val = calibrate_px(q, mb[si_], md[si_], F.t, mr[si_]);
        } else if (SRC == SRC_F32) {
          val = __ldg((const float*)F.src + goff[i]);
        } else {
          val = __half2float(((const __half*)F.src)[goff[i]]);
        }
        v[si_] = val;
      }
    }
    __syncthreads();
    // 2. rows: 2 tasks per window row, 34 outputs each
    if (tid < 2 * kPrefW) {
      const int r = tid >> 1, e0 = (tid & 1) * kPrefRowSeg;
      const float* row = v + r * kPrefWS + e0;  // window col e0 + j <-> ext col e0 + j - 16
      float yp[kPrefRowSeg];
      float y = 0.0f;
#pragma unroll
      for (int j = 0; j < kPrefHalo; ++j) y = __fmaf_rn(kZ1, y, row[j]);
#pragma unroll
      for (int j = 0; j < kPrefRowSeg; ++j) {
        y = __fmaf_rn(kZ1, y, row[kPrefHalo + j]);
        yp[j] = y;
      }
      float ym = 0.0f;
#pragma unroll
      for (int j = kPrefRowSeg + 2 * kPrefHalo - 1; j >= kPrefRowSeg + kPrefHalo; --j)
        ym = __fmaf_rn(kZ1, ym, row[j]);
#pragma unroll
      for (int j = kPrefRowSeg - 1; j >= 0; --j) {
        const float vj = row[kPrefHalo + j];
        ym = __fmaf_rn(kZ1, ym, vj);
        R[r * kPrefRS + e0 + j] = __fmul_rn(kSqrt3, __fsub_rn(__fadd_rn(yp[j], ym), vj));
      }
    }
    __syncthreads();
    // 3. columns: 4 tasks per ext column, 17 outputs each, straight to HBM
    if (tid < 4 * kPrefExt) {
      const int c = tid % kPrefExt, e0 = (tid / kPrefExt) * kPrefColSeg;
      const float* col = R + e0 * kPrefRS + c;  // window row e0 + j <-> ext row e0 + j - 16
      float yp[kPrefColSeg];
      float y = 0.0f;
#pragma unroll
      for (int j = 0; j < kPrefHalo; ++j) y = __fmaf_rn(kZ1, y, col[j * kPrefRS]);
#pragma unroll
      for (int j = 0; j < kPrefColSeg; ++j) {
        y = __fmaf_rn(kZ1, y, col[(kPrefHalo + j) * kPrefRS]);
        yp[j] = y;
      }
      float ym = 0.0f;
#pragma unroll
      for (int j = kPrefColSeg + 2 * kPrefHalo - 1; j >= kPrefColSeg + kPrefHalo; --j)
        ym = __fmaf_rn(kZ1, ym, col[j * kPrefRS]);
      const int gx = x0 - 2 + c;
      float* out = F.coef;
#pragma unroll
      for (int j = kPrefColSeg - 1; j >= 0; --j) {
        const float rj = col[(kPrefHalo + j) * kPrefRS];
        ym = __fmaf_rn(kZ1, ym, rj);
        const int gy = y0 - 2 + e0 + j;
        if (gx >= ox0 && gx < ox1 && gy >= oy0 && gy < oy1)
          out[(int64_t)(gy + 2) * S.coef_pitch + (gx + 2)] =
              __fmul_rn(kSqrt3, __fsub_rn(__fadd_rn(yp[j], ym), rj));
      }
    }
  }
}

}  // namespace irp

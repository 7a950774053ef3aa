// reduce_tile.cuh -- the fused reduction of one output tile of one frame set.
//
// For every frame k of the set (Sec. 2.1 order: calibration, alignment,
// co-adding):
//   1. stage: the frame's source window for this tile is loaded once from HBM,
//      calibrated in FP32, v = (raw - bias - dark*t) * (flat_norm / flat), and
//      stored in shared memory (raw source), or the window of the frame's
//      spline coefficients is loaded (coefficient source);
//   2. sample: each thread resamples its two output pixels with the frame's
//      stencil (nearest, bilinear, 4x4 cubic B-spline) and stores the sample
//      (or +inf when invalid) into the tile's sample array in shared memory.
// Then every thread combines the samples of two output pixels (combine.cuh).
#pragma once

#include "combine.cuh"
#include "common.cuh"

namespace irp {

__device__ __forceinline__ PlanView make_view(const InlinePlan& inl, const void* plan_dev) {
  PlanView v;
  if (plan_dev) {
    const uint8_t* b = (const uint8_t*)plan_dev;
    v.h = (const PlanHeader*)b;
    v.sets = (const SetDesc*)(b + plan_sets_offset());
    v.frames = (const FrameDesc*)(b + plan_frames_offset(v.h->nsets));
  } else {
    v.h = &inl.h;
    v.sets = inl.sets;
    v.frames = inl.frames;
  }
  return v;
}

// flat_norm / flat, latching IRP_ERR_BAD_MASTER for a flat that is not a
// finite positive number.
__device__ __forceinline__ float inv_flat(float flat, float flat_norm, uint32_t* status) {
  if (!(flat > 0.0f) || !isfinite(flat)) {
    latch_status(status, IRP_ERR_BAD_MASTER);
    return __int_as_float(0x7fffffff);
  }
  return __fdiv_rn(flat_norm, flat);
}

__device__ __forceinline__ float calibrate_px(uint16_t raw, float bias, float dark, float t,
                                              float rf) {
  // (raw - bias) - dark*t, then times the reciprocal flat
  const float s = __fmaf_rn(-dark, t, __fsub_rn((float)raw, bias));
  return __fmul_rn(s, rf);
}

template <int STENCIL>
struct StencilShape {
  static constexpr int taps = STENCIL == ST_BSPLINE ? 4 : (STENCIL == ST_BILINEAR ? 2 : 1);
};

// Loads the union window of the masters for this tile (all frames' taps).
__device__ __forceinline__ void stage_masters(const SetDesc& S, int tx0, int ty0, float flat_norm,
                                              float* s_mast, uint32_t* status) {
  const int mw = S.mwin_w, mh = S.mwin_h, mstride = mw;
  float* sb = s_mast;
  float* sd = s_mast + mw * mh;
  float* sr = s_mast + 2 * mw * mh;
  const int gx0 = tx0 + S.mox, gy0 = ty0 + S.moy;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = warp; r < mh; r += kThreads / 32) {
    const int gy = gy0 + r;
    for (int c = lane; c < mw; c += 32) {
      const int gx = gx0 + c;
      float b = 0.0f, d = 0.0f, rf = 0.0f;
      if (gx >= 0 && gx < S.W && gy >= 0 && gy < S.H) {
        const int64_t m = (int64_t)gy * S.master_pitch + gx;
        b = __ldg(S.bias + m);
        d = __ldg(S.dark + m);
        rf = inv_flat(__ldg(S.flat + m), flat_norm, status);
      }
      sb[r * mstride + c] = b;
      sd[r * mstride + c] = d;
      sr[r * mstride + c] = rf;
    }
  }
}

// Stage one frame's calibrated source window (raw source).
template <int STENCIL>
__device__ __forceinline__ void stage_raw(const SetDesc& S, const FrameDesc& F, int tx0, int ty0,
                                          float flat_norm, const float* s_mast, float* s_win,
                                          uint32_t* status) {
  constexpr int T = StencilShape<STENCIL>::taps;
  const int ww = kTW + T - 1, wh = kTH + T - 1;
  const int gx0 = tx0 + F.ox, gy0 = ty0 + F.oy;
  const uint16_t* raw = (const uint16_t*)F.src;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool uni = S.mwin_w > 0;
  const int mw = S.mwin_w, mh = S.mwin_h;
  const int mx = F.ox - S.mox, my = F.oy - S.moy;  // window origin inside the union
  const float t = F.t;
  for (int r = warp; r < wh; r += kThreads / 32) {
    const int gy = gy0 + r;
    for (int c = lane; c < ww; c += 32) {
      const int gx = gx0 + c;
      float v = 0.0f;
      if (gx >= 0 && gx < S.W && gy >= 0 && gy < S.H) {
        const uint16_t q = __ldg(raw + (int64_t)gy * S.src_pitch + gx);
        float b, d, rf;
        if (uni) {
          const int o = (r + my) * mw + (c + mx);
          b = s_mast[o];
          d = s_mast[mw * mh + o];
          rf = s_mast[2 * mw * mh + o];
        } else {
          const int64_t m = (int64_t)gy * S.master_pitch + gx;
          b = __ldg(S.bias + m);
          d = __ldg(S.dark + m);
          rf = inv_flat(__ldg(S.flat + m), flat_norm, status);
        }
        v = calibrate_px(q, b, d, t, rf);
      }
      s_win[r * kWinStride + c] = v;
    }
  }
}

// Stage one frame's window of spline coefficients (mirror-extended).
__device__ __forceinline__ void stage_coef(const SetDesc& S, const FrameDesc& F, int tx0, int ty0,
                                           float* s_win) {
  const int ww = kTW + 3, wh = kTH + 3;
  const int gx0 = tx0 + F.ox, gy0 = ty0 + F.oy;
  const float* cf = F.coef;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int W = S.W, H = S.H;
  for (int r = warp; r < wh; r += kThreads / 32) {
    const int gy = mirror_index(gy0 + r, H);
    for (int c = lane; c < ww; c += 32) {
      const int gx = mirror_index(gx0 + c, W);
      s_win[r * kWinStride + c] = __ldg(cf + (int64_t)gy * W + gx);
    }
  }
}

// Resample this thread's two output pixels (rows 2w, 2w+1 of column lane).
template <int STENCIL>
__device__ __forceinline__ void sample_pair(const FrameDesc& F, const float* s_win, float& a0,
                                            float& a1) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r0 = 2 * warp;
  if (STENCIL == ST_NEAREST) {
    a0 = s_win[r0 * kWinStride + lane];
    a1 = s_win[(r0 + 1) * kWinStride + lane];
  } else if (STENCIL == ST_BILINEAR) {
    const float fx = F.fx, fy = F.fy;
    float h[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float p0 = s_win[(r0 + q) * kWinStride + lane];
      const float p1 = s_win[(r0 + q) * kWinStride + lane + 1];
      h[q] = __fmaf_rn(fx, __fsub_rn(p1, p0), p0);
    }
    a0 = __fmaf_rn(fy, __fsub_rn(h[1], h[0]), h[0]);
    a1 = __fmaf_rn(fy, __fsub_rn(h[2], h[1]), h[1]);
  } else {
    float h[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const float* row = s_win + (r0 + q) * kWinStride + lane;
      float acc = F.wx[0] * row[0];
      acc = __fmaf_rn(F.wx[1], row[1], acc);
      acc = __fmaf_rn(F.wx[2], row[2], acc);
      h[q] = __fmaf_rn(F.wx[3], row[3], acc);
    }
    float acc0 = F.wy[0] * h[0], acc1 = F.wy[0] * h[1];
#pragma unroll
    for (int j = 1; j < 4; ++j) {
      acc0 = __fmaf_rn(F.wy[j], h[j], acc0);
      acc1 = __fmaf_rn(F.wy[j], h[j + 1], acc1);
    }
    a0 = acc0;
    a1 = acc1;
  }
}

template <int NMAX, int STENCIL, int SRC>
__device__ __forceinline__ void reduce_tile(const PlanView& P, int item, float* smem) {
  const PlanHeader& h = *P.h;
  const int si = find_set(P.sets, h.nsets, item);
  const SetDesc& S = P.sets[si];
  const int tile = item - S.tile0;
  const int tx0 = (tile % S.tiles_x) * kTW;
  const int ty0 = (tile / S.tiles_x) * kTH;
  float* s_samples = smem;                          // [n][kTilePx]
  float* s_win = smem + h.smem_samples;             // [kWinRows][kWinStride]
  float* s_mast = s_win + kWinRows * kWinStride;    // [3][mwin_h][mwin_w]
  const int n = S.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int x = tx0 + lane;
  const int y0 = ty0 + 2 * warp, y1 = y0 + 1;

  if (S.ready_flag) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) s_ok = wait_ready(S.ready_flag, S.ready_value, h.spin_limit, h.status);
    __syncthreads();
    if (!s_ok) return;  // status latched; outputs of this tile are left untouched
  }
  float flat_norm = 1.0f;
  if (SRC == SRC_RAW && S.flat_sum) flat_norm = (float)(*S.flat_sum / ((double)S.W * S.H));
  if (SRC == SRC_RAW && S.mwin_w > 0) {
    stage_masters(S, tx0, ty0, flat_norm, s_mast, h.status);
    __syncthreads();
  }
  const float kInf = __int_as_float(0x7f800000);
  for (int k = 0; k < n; ++k) {
    const FrameDesc& F = P.frames[S.frame0 + k];
    if (SRC == SRC_RAW)
      stage_raw<STENCIL>(S, F, tx0, ty0, flat_norm, s_mast, s_win, h.status);
    else
      stage_coef(S, F, tx0, ty0, s_win);
    __syncthreads();
    float a0, a1;
    sample_pair<STENCIL>(F, s_win, a0, a1);
    const bool xv = (x >= F.vx0) & (x <= F.vx1);
    const bool v0 = xv & (y0 >= F.vy0) & (y0 <= F.vy1);
    const bool v1 = xv & (y1 >= F.vy0) & (y1 <= F.vy1);
    a0 = v0 ? a0 : kInf;
    a1 = v1 ? a1 : kInf;
    s_samples[k * kTilePx + (2 * warp) * kTW + lane] = a0;
    s_samples[k * kTilePx + (2 * warp + 1) * kTW + lane] = a1;
    if (S.stack_out && x < S.W) {
      const float qnan = __int_as_float(0x7fc00000);
      if (y0 < S.H) S.stack_out[((int64_t)k * S.H + y0) * S.out_pitch + x] = v0 ? a0 : qnan;
      if (y1 < S.H) S.stack_out[((int64_t)k * S.H + y1) * S.out_pitch + x] = v1 ? a1 : qnan;
    }
    __syncthreads();
  }
  const ClipArgs ca{h.kappa_lo, h.kappa_hi, h.max_iter, h.center, h.ddof};
#pragma unroll 1
  for (int p = threadIdx.x; p < kTilePx; p += kThreads) {
    const int px = tx0 + (p & (kTW - 1)), py = ty0 + p / kTW;
    float s[NMAX];
    int m = 0;
#pragma unroll
    for (int j = 0; j < NMAX; ++j) {
      s[j] = (j < n) ? s_samples[j * kTilePx + p] : kInf;
      m += (s[j] < kInf) ? 1 : 0;
    }
    sort_network<NMAX>(s);
    const CombineOut o = combine_sorted<NMAX>(s, m, ca);
    if (px < S.W && py < S.H) {
      const int64_t oi = (int64_t)py * S.out_pitch + px;
      if (S.mean_out) S.mean_out[oi] = o.mean;
      if (S.median_out) S.median_out[oi] = o.median;
      if (S.nkept_out) S.nkept_out[oi] = (uint16_t)o.kept;
    }
  }
  __syncthreads();
}

}  // namespace irp

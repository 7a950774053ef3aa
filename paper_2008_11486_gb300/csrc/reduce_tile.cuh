// reduce_tile.cuh -- the fused reduction of one output tile of one frame set.
//
// A CTA owns one output tile of one set; each of its 8 warps owns a strip of
// PY output rows and runs its own loop over the set's frames, with no
// CTA-wide barrier inside the loop:
//   1. stage: the strip's source window of frame k + S-1 is copied from HBM
//      into a per-warp shared-memory ring of S stages with cp.async (16-byte
//      chunks, zero-filled outside the frame), so S-1 frames are in flight
//      while frame k is computed;
//   2. calibrate (raw source): lane l holds source column l of the window and
//      computes v = ((raw - bias) - dark*t) * (flat_norm/flat) in registers,
//      the masters coming from a union window in shared memory that is loaded
//      once per tile (Sec. 2.1 calibration);
//   3. resample: the stencil's horizontal taps come from the neighbouring
//      lanes by warp shuffles, the vertical taps from the lane's own rows
//      (nearest, bilinear, or the 4x4 cubic B-spline on spline coefficients);
//   4. the sample (or +inf when invalid) is stored in the tile's sample array.
// After the last frame each lane combines its PY pixels (combine.cuh).
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

// uint16 -> float without the conversion unit: the bits of 2^23 + q.
__device__ __forceinline__ float u16_to_float(uint32_t q) {
  return __fsub_rn(__int_as_float(0x4B000000u | q), 8388608.0f);
}

__device__ __forceinline__ float calibrate_px(uint16_t raw, float bias, float dark, float t,
                                              float rf) {
  // (raw - bias) - dark*t, then times flat_norm/flat
  const float s = __fmaf_rn(-dark, t, __fsub_rn(u16_to_float(raw), bias));
  return __fmul_rn(s, rf);
}

// ------------------------------------------------------------------ cp.async
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------- geometry
template <int STENCIL>
struct StencilShape {
  static constexpr int taps = STENCIL == ST_BSPLINE ? 4 : (STENCIL == ST_BILINEAR ? 2 : 1);
  // output columns per tile: lane l needs source columns l .. l + taps - 1
  static constexpr int tw = 33 - taps;
};

template <int NMAX>
struct RowsPerWarp {
  static constexpr int value = NMAX <= 16 ? 4 : 2;
};

constexpr int kStages = 4;           // cp.async ring depth (frames in flight)
constexpr int kRawChunks = 5;        // 16-byte chunks per staged raw row (40 uint16)
constexpr int kCoefChunks = 9;       // 16-byte chunks per staged coefficient row (36 floats)

template <int SRC, int STENCIL, int PY>
struct StageShape {
  static constexpr int rows = PY + StencilShape<STENCIL>::taps - 1;
  static constexpr int chunks = SRC == SRC_RAW ? kRawChunks : kCoefChunks;
  static constexpr int elems = chunks * (SRC == SRC_RAW ? 8 : 4);  // per row
  static constexpr int bytes = rows * chunks * 16;                  // per stage
};

// Shared memory per CTA of the fused kernel (host helper mirrors this).
__host__ __device__ inline size_t fused_smem_bytes(int src, int stencil, int py, int max_n,
                                                   int mwin_w, int mwin_h) {
  const int taps = stencil == ST_BSPLINE ? 4 : (stencil == ST_BILINEAR ? 2 : 1);
  const int rows = py + taps - 1;
  const int chunks = src == SRC_RAW ? kRawChunks : kCoefChunks;
  const size_t stage = (size_t)kStages * rows * chunks * 16 * (kThreads / 32);
  const size_t samples = (size_t)max_n * (8 * py) * 32 * sizeof(float);
  const size_t masters = (size_t)mwin_w * mwin_h * sizeof(float4);
  const size_t descs = (size_t)max_n * sizeof(FrameDesc);
  return samples + stage + masters + descs;
}

// ------------------------------------------------------------------ staging
// Copies the warp's window of frame F into one stage: rows [gy0, gy0+rows),
// 16-byte chunks from the aligned column xa.  Chunks outside the frame are
// zero-filled; the frames of the raw source must be 16-byte aligned with a
// pitch of a multiple of 8 elements, otherwise every lane copies elements.
template <int SRC, int STENCIL, int PY>
__device__ __forceinline__ void issue_stage(const SetDesc& S, const FrameDesc& F, int gx0, int gy0,
                                            uint8_t* stage, int lane) {
  using SS = StageShape<SRC, STENCIL, PY>;
  if (SRC == SRC_RAW) {
    const uint16_t* base = (const uint16_t*)F.src;
    const int xa = gx0 & ~7;
    if (F.flags & 1) {
      for (int c = lane; c < SS::rows * kRawChunks; c += 32) {
        const int r = c / kRawChunks, j = c - r * kRawChunks;
        const int x = xa + 8 * j, y = gy0 + r;
        int bytes = 0;
        const uint16_t* src = base;
        if (y >= 0 && y < S.H && x >= 0 && x < S.W) {
          bytes = min(16, 2 * (S.W - x));
          src = base + (int64_t)y * S.src_pitch + x;
        }
        cp_async16(stage + (r * kRawChunks + j) * 16, src, bytes);
      }
    } else {
      uint16_t* dst = (uint16_t*)stage;
      for (int e = lane; e < SS::rows * SS::elems; e += 32) {
        const int r = e / SS::elems, i = e - r * SS::elems;
        const int x = xa + i, y = gy0 + r;
        dst[e] = (y >= 0 && y < S.H && x >= 0 && x < S.W) ? base[(int64_t)y * S.src_pitch + x]
                                                           : (uint16_t)0;
      }
    }
  } else {
    // padded coefficient frame: element (x, y) at ((y + 2) * pitch + x + 2)
    const float* base = F.coef;
    const int px = gx0 + 2, py = gy0 + 2;
    const int xa = px & ~3;
    const int Hp = S.H + 4;
    for (int c = lane; c < SS::rows * kCoefChunks; c += 32) {
      const int r = c / kCoefChunks, j = c - r * kCoefChunks;
      const int x = xa + 4 * j, y = py + r;
      int bytes = 0;
      const float* src = base;
      if (y >= 0 && y < Hp && x >= 0 && x < (int)S.coef_pitch) {
        bytes = 16;
        src = base + (int64_t)y * S.coef_pitch + x;
      }
      cp_async16(stage + (r * kCoefChunks + j) * 16, src, bytes);
    }
  }
}

// Loads the union window of the masters for this tile as {bias, dark, rf}.
__device__ __forceinline__ void stage_masters(const SetDesc& S, int tx0, int ty0, float flat_norm,
                                              float4* s_mast, uint32_t* status) {
  const int mw = S.mwin_w, mh = S.mwin_h;
  const int gx0 = tx0 + S.mox, gy0 = ty0 + S.moy;
  for (int e = threadIdx.x; e < mw * mh; e += kThreads) {
    const int r = e / mw, c = e - r * mw;
    const int gx = gx0 + c, gy = gy0 + r;
    float4 m = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (gx >= 0 && gx < S.W && gy >= 0 && gy < S.H) {
      const int64_t o = (int64_t)gy * S.master_pitch + gx;
      m.x = __ldg(S.bias + o);
      m.y = __ldg(S.dark + o);
      m.z = inv_flat(__ldg(S.flat + o), flat_norm, status);
    }
    s_mast[e] = m;
  }
}

template <int NMAX, int STENCIL, int SRC>
__device__ __forceinline__ void reduce_tile(const PlanView& P, int item, float* smem) {
  constexpr int PY = RowsPerWarp<NMAX>::value;
  constexpr int TH = 8 * PY;
  constexpr int TW = StencilShape<STENCIL>::tw;
  constexpr int T = StencilShape<STENCIL>::taps;
  using SS = StageShape<SRC, STENCIL, PY>;
  const PlanHeader& h = *P.h;
  const int si = find_set(P.sets, h.nsets, item);
  const SetDesc& S = P.sets[si];
  const int tile = item - S.tile0;
  const int tx0 = (tile % S.tiles_x) * TW;
  const int ty0 = (tile / S.tiles_x) * TH;
  const int n = S.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wy0 = ty0 + warp * PY;  // first output row of this warp
  const int x = tx0 + lane;

  float* s_samples = smem;                                    // [n][TH][32]
  uint8_t* s_stage = (uint8_t*)(smem + h.smem_samples) + warp * kStages * SS::bytes;
  float4* s_mast = (float4*)((uint8_t*)(smem + h.smem_samples) +
                             (size_t)kStages * SS::bytes * (kThreads / 32));
  FrameDesc* s_desc = (FrameDesc*)(s_mast + h.smem_master);  // the set's frames

  if (S.ready_flag) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) s_ok = wait_ready(S.ready_flag, S.ready_value, h.spin_limit, h.status);
    __syncthreads();
    if (!s_ok) return;  // status latched; this tile's outputs are left untouched
  }
  {
    // frame descriptors of the set: one copy per tile, read from shared memory
    const uint4* src = (const uint4*)(P.frames + S.frame0);
    uint4* dst = (uint4*)s_desc;
    for (int i = threadIdx.x; i < n * (int)(sizeof(FrameDesc) / 16); i += kThreads) dst[i] = src[i];
  }
  float flat_norm = 1.0f;
  if (SRC == SRC_RAW && S.flat_sum) flat_norm = (float)(*S.flat_sum / ((double)S.W * S.H));
  if (SRC == SRC_RAW && S.mwin_w > 0) stage_masters(S, tx0, ty0, flat_norm, s_mast, h.status);
  __syncthreads();

  const FrameDesc* frames = s_desc;
  // prologue: frames 0 .. kStages-2 in flight
#pragma unroll
  for (int k = 0; k < kStages - 1; ++k) {
    if (k < n) {
      const FrameDesc& F = frames[k];
      issue_stage<SRC, STENCIL, PY>(S, F, tx0 + F.ox, wy0 + F.oy, s_stage + k * SS::bytes, lane);
    }
    cp_async_commit();
  }
  const float kInf = __int_as_float(0x7f800000);
  const float qnan = __int_as_float(0x7fc00000);
  for (int k = 0; k < n; ++k) {
    cp_async_wait<kStages - 2>();
    __syncwarp();
    {
      const int kn = k + kStages - 1;
      if (kn < n) {
        const FrameDesc& Fn = frames[kn];
        issue_stage<SRC, STENCIL, PY>(S, Fn, tx0 + Fn.ox, wy0 + Fn.oy,
                                      s_stage + (kn % kStages) * SS::bytes, lane);
      }
      cp_async_commit();
    }
    const FrameDesc& F = frames[k];
    const uint8_t* st = s_stage + (k % kStages) * SS::bytes;
    float v[SS::rows];
    if (SRC == SRC_RAW) {
      const int off = (tx0 + F.ox) & 7;
      const uint16_t* raw = (const uint16_t*)st;
      const float t = F.t;
      if (S.mwin_w > 0) {
        const int mrow = warp * PY + (F.oy - S.moy), mcol = lane + (F.ox - S.mox);
#pragma unroll
        for (int r = 0; r < SS::rows; ++r) {
          const float4 m = s_mast[(mrow + r) * S.mwin_w + mcol];
          v[r] = calibrate_px(raw[r * SS::elems + lane + off], m.x, m.y, t, m.z);
        }
      } else {  // offsets too spread for a union window: masters from global memory
        const int gx = tx0 + F.ox + lane;
#pragma unroll
        for (int r = 0; r < SS::rows; ++r) {
          const int gy = wy0 + F.oy + r;
          float b = 0.0f, d = 0.0f, rf = 0.0f;
          if (gx >= 0 && gx < S.W && gy >= 0 && gy < S.H) {
            const int64_t o = (int64_t)gy * S.master_pitch + gx;
            b = __ldg(S.bias + o);
            d = __ldg(S.dark + o);
            rf = inv_flat(__ldg(S.flat + o), flat_norm, h.status);
          }
          v[r] = calibrate_px(raw[r * SS::elems + lane + off], b, d, t, rf);
        }
      }
    } else {
      const int off = (tx0 + F.ox + 2) & 3;
      const float* cf = (const float*)st;
#pragma unroll
      for (int r = 0; r < SS::rows; ++r) v[r] = cf[r * SS::elems + lane + off];
    }
    float a[PY];
    if (STENCIL == ST_NEAREST) {
#pragma unroll
      for (int q = 0; q < PY; ++q) a[q] = v[q];
    } else if (STENCIL == ST_BILINEAR) {
      float hrow[SS::rows];
#pragma unroll
      for (int r = 0; r < SS::rows; ++r) {
        const float p1 = __shfl_down_sync(0xffffffffu, v[r], 1);
        hrow[r] = __fmaf_rn(F.fx, __fsub_rn(p1, v[r]), v[r]);
      }
#pragma unroll
      for (int q = 0; q < PY; ++q) a[q] = __fmaf_rn(F.fy, __fsub_rn(hrow[q + 1], hrow[q]), hrow[q]);
    } else {
      const float w0 = F.wx[0], w1 = F.wx[1], w2 = F.wx[2], w3 = F.wx[3];
      float hrow[SS::rows];
#pragma unroll
      for (int r = 0; r < SS::rows; ++r) {
        const float p1 = __shfl_down_sync(0xffffffffu, v[r], 1);
        const float p2 = __shfl_down_sync(0xffffffffu, v[r], 2);
        const float p3 = __shfl_down_sync(0xffffffffu, v[r], 3);
        float acc = w0 * v[r];
        acc = __fmaf_rn(w1, p1, acc);
        acc = __fmaf_rn(w2, p2, acc);
        hrow[r] = __fmaf_rn(w3, p3, acc);
      }
#pragma unroll
      for (int q = 0; q < PY; ++q) {
        float acc = F.wy[0] * hrow[q];
        acc = __fmaf_rn(F.wy[1], hrow[q + 1], acc);
        acc = __fmaf_rn(F.wy[2], hrow[q + 2], acc);
        a[q] = __fmaf_rn(F.wy[3], hrow[q + 3], acc);
      }
    }
    const bool xv = (x >= F.vx0) & (x <= F.vx1);
    float* sk = s_samples + ((size_t)k * TH + warp * PY) * 32 + lane;
#pragma unroll
    for (int q = 0; q < PY; ++q) {
      const int y = wy0 + q;
      const bool ok = xv & (y >= F.vy0) & (y <= F.vy1);
      sk[q * 32] = ok ? a[q] : kInf;
      if (S.stack_out && lane < TW && x < S.W && y < S.H)
        S.stack_out[((int64_t)k * S.H + y) * S.out_pitch + x] = ok ? a[q] : qnan;
    }
  }
  cp_async_wait<0>();
  __syncwarp();
  (void)T;

  const ClipArgs ca{h.kappa_lo, h.kappa_hi, h.max_iter, h.center, h.ddof};
  if (lane < TW && x < S.W) {
#pragma unroll 1
    for (int q = 0; q < PY; ++q) {
      const int y = wy0 + q;
      if (y >= S.H) break;
      const float* sp = s_samples + (size_t)(warp * PY + q) * 32 + lane;
      float s[NMAX];
      int m = 0;
#pragma unroll
      for (int j = 0; j < NMAX; ++j) {
        s[j] = (j < n) ? sp[(size_t)j * TH * 32] : kInf;
        m += (s[j] < kInf) ? 1 : 0;
      }
      sort_network<NMAX>(s);
      const CombineOut o = combine_sorted<NMAX>(s, m, ca);
      const int64_t oi = (int64_t)y * S.out_pitch + x;
      if (S.mean_out) S.mean_out[oi] = o.mean;
      if (S.median_out) S.median_out[oi] = o.median;
      if (S.nkept_out) S.nkept_out[oi] = (uint16_t)o.kept;
    }
  }
  __syncthreads();  // descriptors and union window are reused by the next tile
}

}  // namespace irp

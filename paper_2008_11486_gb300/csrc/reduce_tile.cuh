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

// Output rows per warp (tile height / 8): the two choices of each register
// bucket (the autotuner picks one; the first is the default).
__host__ __device__ constexpr int rows_per_warp_default(int nmax) { return nmax <= 16 ? 4 : 2; }
__host__ __device__ constexpr int rows_per_warp_alt(int nmax) { return nmax <= 16 ? 2 : 1; }

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
// What the frame loop needs of one frame for the current tile, built once per
// tile in shared memory (128 bytes).
struct FrameRec {
  const uint8_t* base;   // staging source: element (ybase, xa) of the frame
  const uint8_t* fbase;  // a valid address inside the frame (zero-byte copies)
  int ybase, xa;         // first staged row / aligned first staged column
  int off;               // tile's first source column inside the staged row
  int mofs;              // union-window offset of the tile's first source pixel
  int ox, oy;            // tap origin (masters read from global memory)
  float fx, fy, t;
  int vx0, vx1, vy0, vy1;
  int flags;
  float wx[4], wy[4];
  int pad[6];
};
static_assert(sizeof(FrameRec) == 128, "FrameRec layout");

template <int SRC>
__device__ __forceinline__ FrameRec make_rec(const FrameDesc& F, int tx0, int ty0, int64_t pitch,
                                             int mox, int moy, int mwin_w) {
  FrameRec R;
  const int gx0 = tx0 + F.ox, gy0 = ty0 + F.oy;
  if (SRC == SRC_RAW) {
    R.xa = gx0 & ~7;
    R.off = gx0 - R.xa;
    R.ybase = gy0;
    R.fbase = (const uint8_t*)F.src;
    R.base = R.fbase + ((int64_t)gy0 * pitch + R.xa) * 2;
  } else {  // padded coefficient frame: element (x, y) at ((y + 2) * pitch + x + 2)
    R.xa = (gx0 + 2) & ~3;
    R.off = gx0 + 2 - R.xa;
    R.ybase = gy0 + 2;
    R.fbase = (const uint8_t*)F.coef;
    R.base = R.fbase + ((int64_t)R.ybase * pitch + R.xa) * 4;
  }
  R.mofs = (F.oy - moy) * mwin_w + (F.ox - mox);
  R.ox = F.ox;
  R.oy = F.oy;
  R.fx = F.fx;
  R.fy = F.fy;
  R.t = F.t;
  R.vx0 = F.vx0;
  R.vx1 = F.vx1;
  R.vy0 = F.vy0;
  R.vy1 = F.vy1;
  R.flags = F.flags;
  for (int i = 0; i < 4; ++i) {
    R.wx[i] = F.wx[i];
    R.wy[i] = F.wy[i];
  }
  return R;
}

// Copies the warp's window of one frame into one stage.  Each lane owns up
// to kIt fixed 16-byte chunks of the window (row delta, column delta and byte
// offset precomputed per tile); chunks outside the frame are zero-filled.  Raw
// frames that are not 16-byte aligned with a pitch of 8k elements are copied
// element by element instead.
template <int SRC, int kIt>
struct LaneChunks {
  int drow[kIt], dcol[kIt], soff[kIt];
  int64_t goff[kIt];
};

template <int SRC, int STENCIL, int PY>
__device__ __forceinline__ void issue_stage(const FrameRec& R, const LaneChunks<SRC, (StageShape<SRC, STENCIL, PY>::rows * StageShape<SRC, STENCIL, PY>::chunks + 31) / 32>& L,
                                            int Hlim, int Wlim, int64_t pitch, uint8_t* stage,
                                            int lane, int wrow) {
  using SS = StageShape<SRC, STENCIL, PY>;
  constexpr int kIt = (SS::rows * SS::chunks + 31) / 32;
  if (SRC == SRC_RAW && !(R.flags & 1)) {
    uint16_t* dst = (uint16_t*)stage;
    const uint16_t* fb = (const uint16_t*)R.fbase;
    for (int e = lane; e < SS::rows * SS::elems; e += 32) {
      const int r = e / SS::elems, i = e - r * SS::elems;
      const int y = R.ybase + wrow + r, xx = R.xa + i;
      dst[e] = ((unsigned)y < (unsigned)Hlim && (unsigned)xx < (unsigned)Wlim)
                   ? fb[(int64_t)y * pitch + xx] : (uint16_t)0;
    }
    return;
  }
#pragma unroll
  for (int it = 0; it < kIt; ++it) {
    if (L.soff[it] < 0) continue;
    const int y = R.ybase + L.drow[it], xx = R.xa + L.dcol[it];
    int bytes = 0;
    const uint8_t* src = R.fbase;
    if ((unsigned)y < (unsigned)Hlim && (unsigned)xx < (unsigned)Wlim) {
      bytes = SRC == SRC_RAW ? min(16, 2 * (Wlim - xx)) : 16;
      src = R.base + L.goff[it];
    }
    cp_async16(stage + L.soff[it], src, bytes);
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

template <int NMAX, int STENCIL, int SRC, int PY>
__device__ __forceinline__ void reduce_tile(const PlanView& P, int item, float* smem) {
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
  // set fields used inside the frame loop, in registers
  const int W = S.W, H = S.H;
  const int mwin_w = S.mwin_w;
  float* const stack_out = S.stack_out;
  const int64_t out_pitch = S.out_pitch;
  const int64_t pitch = SRC == SRC_RAW ? S.src_pitch : S.coef_pitch;
  const int Hlim = SRC == SRC_RAW ? H : H + 4;
  const int Wlim = SRC == SRC_RAW ? W : (int)S.coef_pitch;

  float* s_samples = smem;                                    // [n][TH][32]
  uint8_t* s_stage = (uint8_t*)(smem + h.smem_samples) + warp * kStages * SS::bytes;
  float4* s_mast = (float4*)((uint8_t*)(smem + h.smem_samples) +
                             (size_t)kStages * SS::bytes * (kThreads / 32));
  FrameRec* s_rec = (FrameRec*)(s_mast + h.smem_master);    // the set's frames

  if (S.ready_flag) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) s_ok = wait_ready(S.ready_flag, S.ready_value, h.spin_limit, h.status);
    __syncthreads();
    if (!s_ok) return;  // status latched; this tile's outputs are left untouched
  }
  for (int k = threadIdx.x; k < n; k += kThreads)
    s_rec[k] = make_rec<SRC>(P.frames[S.frame0 + k], tx0, ty0, pitch, S.mox, S.moy, mwin_w);
  float flat_norm = 1.0f;
  if (SRC == SRC_RAW && S.flat_sum) flat_norm = (float)(*S.flat_sum / ((double)S.W * S.H));
  if (SRC == SRC_RAW && S.mwin_w > 0) stage_masters(S, tx0, ty0, flat_norm, s_mast, h.status);
  // this lane's staging chunks (frame-independent)
  constexpr int kIt = (SS::rows * SS::chunks + 31) / 32;
  LaneChunks<SRC, kIt> LC;
#pragma unroll
  for (int it = 0; it < kIt; ++it) {
    const int c = lane + 32 * it;
    const int r = c / SS::chunks, j = c - r * SS::chunks;
    const int colw = SRC == SRC_RAW ? 8 : 4, esz = SRC == SRC_RAW ? 2 : 4;
    LC.drow[it] = warp * PY + r;
    LC.dcol[it] = colw * j;
    LC.soff[it] = c < SS::rows * SS::chunks ? c * 16 : -1;
    LC.goff[it] = ((int64_t)LC.drow[it] * pitch + LC.dcol[it]) * esz;
  }
  __syncthreads();

  const FrameRec* frames = s_rec;
  // prologue: frames 0 .. kStages-2 in flight
#pragma unroll
  for (int k = 0; k < kStages - 1; ++k) {
    if (k < n)
      issue_stage<SRC, STENCIL, PY>(frames[k], LC, Hlim, Wlim, pitch, s_stage + k * SS::bytes,
                                    lane, warp * PY);
    cp_async_commit();
  }
  const float kInf = __int_as_float(0x7f800000);
  const float qnan = __int_as_float(0x7fc00000);
  for (int k = 0; k < n; ++k) {
    cp_async_wait<kStages - 2>();
    __syncwarp();
    {
      const int kn = k + kStages - 1;
      if (kn < n)
        issue_stage<SRC, STENCIL, PY>(frames[kn], LC, Hlim, Wlim, pitch,
                                      s_stage + (kn % kStages) * SS::bytes, lane, warp * PY);
      cp_async_commit();
    }
    const FrameRec& F = frames[k];
    const uint8_t* st = s_stage + (k % kStages) * SS::bytes;
    float v[SS::rows];
    if (SRC == SRC_RAW) {
      const int off = F.off;
      const uint16_t* raw = (const uint16_t*)st;
      const float t = F.t;
      if (mwin_w > 0) {
        const float4* mp = s_mast + F.mofs + warp * PY * mwin_w + lane;
#pragma unroll
        for (int r = 0; r < SS::rows; ++r) {
          const float4 m = mp[r * mwin_w];
          v[r] = calibrate_px(raw[r * SS::elems + lane + off], m.x, m.y, t, m.z);
        }
      } else {  // offsets too spread for a union window: masters from global memory
        const int gx = tx0 + F.ox + lane;
#pragma unroll
        for (int r = 0; r < SS::rows; ++r) {
          const int gy = wy0 + F.oy + r;
          float b = 0.0f, d = 0.0f, rf = 0.0f;
          if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
            const int64_t o = (int64_t)gy * S.master_pitch + gx;
            b = __ldg(S.bias + o);
            d = __ldg(S.dark + o);
            rf = inv_flat(__ldg(S.flat + o), flat_norm, h.status);
          }
          v[r] = calibrate_px(raw[r * SS::elems + lane + off], b, d, t, rf);
        }
      }
    } else {
      const int off = F.off;
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
      if (stack_out && lane < TW && x < W && y < H)
        stack_out[((int64_t)k * H + y) * out_pitch + x] = ok ? a[q] : qnan;
    }
  }
  cp_async_wait<0>();
  __syncwarp();
  (void)T;

  const ClipArgs ca{h.kappa_lo, h.kappa_hi, h.max_iter, h.center, h.ddof};
  float* const mean_out = S.mean_out;
  float* const median_out = S.median_out;
  uint16_t* const nkept_out = S.nkept_out;
  if (lane < TW && x < W) {
#pragma unroll 1
    for (int q = 0; q < PY; ++q) {
      const int y = wy0 + q;
      if (y >= H) break;
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
      const int64_t oi = (int64_t)y * out_pitch + x;
      if (mean_out) mean_out[oi] = o.mean;
      if (median_out) median_out[oi] = o.median;
      if (nkept_out) nkept_out[oi] = (uint16_t)o.kept;
    }
  }
  __syncthreads();  // descriptors and union window are reused by the next tile
}

}  // namespace irp

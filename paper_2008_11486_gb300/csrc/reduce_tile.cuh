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
//      computes v = (raw - (bias + dark*t)) * (flat_norm/flat) in registers,
//      the masters coming from a union window in shared memory that is loaded
//      once per tile (Sec. 2.1 calibration); for a set of one exposure time
//      and no bad-pixel mask the window holds {bias + dark*t, flat_norm/flat}
//      (8 bytes a pixel) instead of {bias, dark, flat_norm/flat, mask};
//   3. resample: the stencil's horizontal taps come from the neighbouring
//      lanes by warp shuffles, the vertical taps from the lane's own rows
//      (nearest, bilinear, Keys' 4x4 cubic convolution, or the 4x4 cubic
//      B-spline on spline coefficients);
//   4. the sample (or +inf when invalid) is stored in the tile's sample array.
// After the last frame each lane combines its PY pixels (combine.cuh).
#pragma once

#include <limits.h>

#include <type_traits>

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

// The two uint16 halves of a 32-bit word as floats: one byte permute builds
// the bits of 2^23 + q.
__device__ __forceinline__ float u16_lo_to_float(uint32_t w) {
  return __fsub_rn(__int_as_float(__byte_perm(w, 0x4B00u, 0x5410u)), 8388608.0f);
}
__device__ __forceinline__ float u16_hi_to_float(uint32_t w) {
  return __fsub_rn(__int_as_float(__byte_perm(w, 0x4B00u, 0x5432u)), 8388608.0f);
}

// Calibration of one pixel: (raw - (bias + dark*t)) * (flat_norm/flat).  The
// level removed from the raw count, bias + dark*t, is one correctly rounded
// fma, so that the frames of one exposure time can share it (the premerged
// master window of the fused kernel gives bit-identical values).
__device__ __forceinline__ float calib_level(float bias, float dark, float t) {
  return __fmaf_rn(dark, t, bias);
}

__device__ __forceinline__ float calibrate_pxf(float rawf, float bias, float dark, float t,
                                               float rf) {
  return __fmul_rn(__fsub_rn(rawf, calib_level(bias, dark, t)), rf);
}

__device__ __forceinline__ float calibrate_px(uint16_t raw, float bias, float dark, float t,
                                              float rf) {
  return calibrate_pxf(u16_to_float(raw), bias, dark, t, rf);
}

// ------------------------------------------------------------------ cp.async
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem),
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
  static constexpr int taps_x =
      (STENCIL == ST_BSPLINE || STENCIL == ST_CUBIC) ? 4 : (STENCIL == ST_BILINEAR ? 2 : 1);
  static constexpr int taps_y =
      (STENCIL == ST_BSPLINE || STENCIL == ST_BSPLINE_V || STENCIL == ST_CUBIC)
          ? 4 : (STENCIL == ST_BILINEAR ? 2 : 1);
  // output columns per tile: lane l needs source columns l .. l + taps_x - 1
  static constexpr int tw = 33 - taps_x;
};

// Output rows per warp (tile height / 8): the two choices of each register
// bucket and stencil (the autotuner picks one; the first is the default).
// Above 40 frames one row per warp lets two CTAs share an SM (half the
// samples in shared memory, at most 128 registers), measured faster for the
// 2-tap and filtered-row stencils on 48 and 64 x 4096^2 sets (3 to 6%); the
// 4-tap Keys stencil, whose single rows stage four source rows each, keeps
// two rows per warp (4 to 8% faster so).
__host__ __device__ constexpr bool tall_tiles(int nmax, int stencil) {
  return nmax <= 40 || stencil == ST_CUBIC || stencil == ST_BSPLINE;
}
__host__ __device__ constexpr int rows_per_warp_default(int nmax, int stencil) {
  return nmax <= 16 ? 4 : (tall_tiles(nmax, stencil) ? 2 : 1);
}
__host__ __device__ constexpr int rows_per_warp_alt(int nmax, int stencil) {
  return nmax <= 16 ? 2 : (tall_tiles(nmax, stencil) ? 1 : 2);
}

// Interior tiles of raw sources with at most 2 output rows per warp take the
// frames two at a time (more independent work per warp between waits).
__host__ __device__ constexpr bool pair_frames(int src, int py) { return src == SRC_RAW && py <= 2; }

// cp.async ring depth: 6 stages when the frames go in pairs (four frames in
// flight while a pair is computed), else 4 (three in flight while a frame is).
__host__ __device__ constexpr int stage_count(int src, int stencil, int py) {
  (void)stencil;
  return pair_frames(src, py) ? 6 : 4;
}
constexpr int kRawChunks = 5;        // 16-byte chunks per staged raw row (40 uint16)
constexpr int kCoefChunks = 9;       // 16-byte chunks per staged coefficient row (36 floats)
constexpr int kRowChunks = 8;        // 16-byte chunks per staged filtered row (32 floats)

__host__ __device__ constexpr int stage_chunks(int src, int stencil) {
  return src == SRC_RAW ? kRawChunks : (stencil == ST_BSPLINE_V ? kRowChunks : kCoefChunks);
}

template <int SRC, int STENCIL, int PY>
struct StageShape {
  static constexpr int rows = PY + StencilShape<STENCIL>::taps_y - 1;
  static constexpr int chunks = stage_chunks(SRC, STENCIL);
  static constexpr int elems = chunks * (SRC == SRC_RAW ? 8 : 4);  // per row
  static constexpr int bytes = rows * chunks * 16;                  // per stage
};

// Frame records per CTA: 144 bytes each (9 x 16), so that the 16-byte stores
// of consecutive records fall into distinct bank groups.
constexpr int kRecBytes = 144;

// Float4 entries reserved for a master union window of w x h pixels: the
// {bias, dark, rf, mask} window (16 bytes a pixel), or, packed, the planar
// copies of the three masters (12 bytes a pixel) that become the premerged
// {bias + dark*t, rf} window (8 bytes a pixel) in place.
__host__ __device__ constexpr int master_window_f4(int w, int h, bool packed) {
  return packed ? (3 * w * h + 3) / 4 : w * h;
}
constexpr int kMaxWindowPx = 4096;  // 64 KB of float4 entries

// Shared memory per CTA of the fused kernel (host helper mirrors this).
__host__ __device__ inline size_t fused_smem_bytes(int src, int stencil, int py, int max_n,
                                                   int mwin_f4) {
  const int taps = (stencil == ST_BSPLINE || stencil == ST_BSPLINE_V || stencil == ST_CUBIC)
                       ? 4 : (stencil == ST_BILINEAR ? 2 : 1);
  const int rows = py + taps - 1;
  const int chunks = stage_chunks(src, stencil);
  const size_t stage = (size_t)stage_count(src, stencil, py) * rows * chunks * 16 * (kThreads / 32);
  const size_t samples = (size_t)max_n * (8 * py) * 32 * sizeof(float);
  const size_t masters = (size_t)mwin_f4 * sizeof(float4);  // master_window_f4 entries
  const size_t descs = (size_t)max_n * kRecBytes;
  return samples + stage + masters + descs;
}

// ------------------------------------------------------------------ staging
// What the frame loop needs of one frame for the current tile, built once per
// tile in shared memory (kRecBytes).  The fields the loop reads every frame
// are grouped into 16-byte vectors, so each group is one broadcast load.
struct FrameRec {
  // compute: tile's first source column inside the staged row, union-window
  // offset of the tile's first source pixel, and the column validity range
  // as (first, width) for one unsigned compare (an empty range has first
  // INT_MIN, which no column reaches)
  int off, mofs, vx0, vxw;
  float fx, fy, t, pad0;
  int vy0, vyw, ox, oy;       // row validity; tap origin for global masters
  float wx[4], wy[4];         // spline weights
  const uint8_t* base;        // staging source: element (ybase, xa) of the frame
  const uint8_t* fbase;       // a valid address inside the frame (zero-byte copies)
  int ybase, xa, flags, last_tap;  // first staged row / aligned first staged column;
                              // FrameDesc::last_tap
  float na, nz;               // per-frame normalisation: sample = fma(sample, na, nz)
  int pad2[6];
};
static_assert(sizeof(FrameRec) == kRecBytes, "FrameRec layout");

// flags: bit 0 = raw frame 16-byte aligned with a pitch of 8k elements;
// bit 1 = the tile's whole staging window (rows x elems from (ybase, xa)) lies
// inside the frame, so its chunks need no bounds checks; bit 2 = every output
// pixel of the tile inside the frame, [tx0, tx1] x [ty0, ty1], has a valid
// sample of this frame.
template <int SRC, int STENCIL>
__device__ __forceinline__ FrameRec make_rec(const FrameDesc& F, int tx0, int ty0, int64_t pitch,
                                             int mox, int moy, int mwin_w, int win_rows,
                                             int win_elems, int Hlim, int Wlim, int tx1,
                                             int ty1) {
  FrameRec R;
  const int gx0 = tx0 + F.ox, gy0 = ty0 + F.oy;
  if (SRC == SRC_RAW) {
    R.xa = gx0 & ~7;
    R.off = gx0 - R.xa;
    R.ybase = gy0;
    R.fbase = (const uint8_t*)F.src;
    R.base = R.fbase + ((int64_t)gy0 * pitch + R.xa) * 2;
  } else if (STENCIL == ST_BSPLINE_V) {
    // filtered rows on the output columns: element (x, y) at ((y + 2) * pitch + x)
    R.xa = tx0;
    R.off = 0;
    R.ybase = gy0 + 2;
    R.fbase = (const uint8_t*)F.coef;
    R.base = R.fbase + ((int64_t)R.ybase * pitch + R.xa) * 4;
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
  R.pad0 = 0.0f;
  const bool ex = F.vx1 < F.vx0, ey = F.vy1 < F.vy0;
  R.vx0 = ex ? INT_MIN : F.vx0;
  R.vxw = ex ? 0 : F.vx1 - F.vx0;
  R.vy0 = ey ? INT_MIN : F.vy0;
  R.vyw = ey ? 0 : F.vy1 - F.vy0;
  const bool aligned_src = SRC != SRC_RAW || (F.flags & 1);
  const bool interior = aligned_src && R.ybase >= 0 && R.ybase + win_rows <= Hlim && R.xa >= 0 &&
                        R.xa + win_elems <= Wlim;
  const bool all_valid = F.vx0 <= tx0 && F.vx1 >= tx1 && F.vy0 <= ty0 && F.vy1 >= ty1;
  R.flags = (F.flags & 1) | (interior ? 2 : 0) | (all_valid ? 4 : 0);
  R.last_tap = F.last_tap;
  for (int i = 0; i < 4; ++i) {
    R.wx[i] = F.wx[i];
    R.wy[i] = F.wy[i];
  }
  R.na = F.norm ? F.norm->na : 1.0f;
  R.nz = F.norm ? F.norm->nz : 0.0f;
  for (int i = 0; i < 6; ++i) R.pad2[i] = 0;
  return R;
}

// v in [lo, lo + w] with one unsigned compare (w >= 0; lo = INT_MIN: never)
__device__ __forceinline__ bool in_range(int v, int lo, int w) {
  return (unsigned)v - (unsigned)lo <= (unsigned)w;
}

// One 16-byte cp.async when p is set, zero-filling the bytes past src_bytes.
__device__ __forceinline__ void cp_async16_if(bool p, void* smem, const void* gmem,
                                              int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.b32 q, %3, 0;\n"
      " @q cp.async.cg.shared.global [%0], [%1], 16, %2;\n}\n" ::"r"(s),
      "l"(gmem), "r"(src_bytes), "r"((int)p)
      : "memory");
}

// Copies the warp's window of one frame into one stage.  Each lane owns up
// to kIt fixed 16-byte chunks of the window (row delta, column delta and byte
// offset precomputed per tile); chunks outside the frame are zero-filled.  Raw
// frames that are not 16-byte aligned with a pitch of 8k elements are copied
// element by element instead.
template <int SRC, int kIt>
struct LaneChunks {
  int drow[kIt], dcol[kIt], soff[kIt];  // soff: stage byte offset (0 when the lane has none)
  bool has[kIt];                        // the lane owns chunk it
  int64_t goff[kIt];
};

template <int SRC, int STENCIL, int PY>
__device__ __forceinline__ void issue_stage(const FrameRec& R, const LaneChunks<SRC, (StageShape<SRC, STENCIL, PY>::rows * StageShape<SRC, STENCIL, PY>::chunks + 31) / 32>& L,
                                            int Hlim, int Wlim, int64_t pitch, uint8_t* stage,
                                            int lane, int wrow) {
  using SS = StageShape<SRC, STENCIL, PY>;
  constexpr int kIt = (SS::rows * SS::chunks + 31) / 32;
  const int4 st = *(const int4*)&R.ybase;  // ybase, xa, flags
  if (SRC == SRC_RAW && !(st.z & 1)) {
    uint16_t* dst = (uint16_t*)stage;
    const uint16_t* fb = (const uint16_t*)R.fbase;
    for (int e = lane; e < SS::rows * SS::elems; e += 32) {
      const int r = e / SS::elems, i = e - r * SS::elems;
      const int y = st.x + wrow + r, xx = st.y + i;
      dst[e] = ((unsigned)y < (unsigned)Hlim && (unsigned)xx < (unsigned)Wlim)
                   ? fb[(int64_t)y * pitch + xx] : (uint16_t)0;
    }
    return;
  }
  const uint8_t* base = R.base;
  if (st.z & 2) {  // window inside the frame: no bounds checks
#pragma unroll
    for (int it = 0; it < kIt; ++it) cp_async16_if(L.has[it], stage + L.soff[it], base + L.goff[it], 16);
    return;
  }
  const uint8_t* fbase = R.fbase;
#pragma unroll
  for (int it = 0; it < kIt; ++it) {
    const int y = st.x + L.drow[it], xx = st.y + L.dcol[it];
    const bool in = ((unsigned)y < (unsigned)Hlim) & ((unsigned)xx < (unsigned)Wlim);
    const int bytes = in ? (SRC == SRC_RAW ? min(16, 2 * (Wlim - xx)) : 16) : 0;
    const uint8_t* src = in ? base + L.goff[it] : fbase;
    cp_async16_if(L.has[it], stage + L.soff[it], src, bytes);
  }
}

// issue_stage for a frame whose window lies inside the frame and is aligned:
// every owned chunk is one unconditional 16-byte copy.
template <int SRC, int kIt>
__device__ __forceinline__ void issue_stage_inside(const FrameRec& R,
                                                   const LaneChunks<SRC, kIt>& L,
                                                   uint8_t* stage) {
  const uint8_t* base = R.base;
#pragma unroll
  for (int it = 0; it < kIt; ++it) cp_async16_if(L.has[it], stage + L.soff[it], base + L.goff[it], 16);
}

// The union window of the masters for this tile.  Unpacked: the three
// masters are copied asynchronously into the float4 slots {bias, dark, rf,
// mask} (zero outside the frame), then finish_masters turns the flat into
// flat_norm/flat and sets the mask flag.  Packed (pk): they are copied into
// three planar arrays, which finish_masters reads and then overwrites with
// the float2 window {bias + dark*t, flat_norm/flat}.
__device__ __forceinline__ void issue_masters(const SetDesc& S, int tx0, int ty0,
                                              float4* s_mast, bool pk) {
  const int mw = S.mwin_w, mh = S.mwin_h, np = mw * mh;
  const int gx0 = tx0 + S.mox, gy0 = ty0 + S.moy;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* const planar = (float*)s_mast;  // bias, dark, flat: np floats each
  for (int r = warp; r < mh; r += kThreads / 32) {
    const int gy = gy0 + r;
    const bool yin = gy >= 0 && gy < S.H;
    for (int c = lane; c < mw; c += 32) {
      const int gx = gx0 + c;
      const bool in = yin && gx >= 0 && gx < S.W;
      const int64_t o = in ? (int64_t)gy * S.master_pitch + gx : 0;
      const int nb = in ? 4 : 0;
      const int e = r * mw + c;
      if (pk) {
        cp_async4(planar + e, S.bias + o, nb);
        cp_async4(planar + np + e, S.dark + o, nb);
        cp_async4(planar + 2 * np + e, S.flat + o, nb);
      } else {
        float* d = (float*)(s_mast + e);
        cp_async4(d + 0, S.bias + o, nb);
        cp_async4(d + 1, S.dark + o, nb);
        cp_async4(d + 2, S.flat + o, nb);
      }
    }
  }
}

// Called by all threads of the CTA after the masters' copies have landed;
// ends with the window complete (a CTA barrier inside).
__device__ __forceinline__ void finish_masters(const SetDesc& S, int tx0, int ty0,
                                               float flat_norm, float4* s_mast, bool pk,
                                               float t, uint32_t* status) {
  const int mw = S.mwin_w, mh = S.mwin_h, np = mw * mh;
  const int gx0 = tx0 + S.mox, gy0 = ty0 + S.moy;
  if (pk) {
    // every thread reads its pixels (threadIdx.x + kThreads * i) into
    // registers, then, after a barrier, writes them to the window in place
    constexpr int kPer = kMaxWindowPx / kThreads;
    const float* const planar = (const float*)s_mast;
    float lv[kPer], rf[kPer];
    // (row, column) of pixel e, stepped by kThreads without divisions
    const int dr = kThreads / mw, dc = kThreads - dr * mw;
    int r = threadIdx.x / mw, c = threadIdx.x - r * mw;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int e = threadIdx.x + kThreads * i;
      lv[i] = rf[i] = 0.0f;
      if (e < np) {
        const int gy = gy0 + r, gx = gx0 + c;
        const bool in = gy >= 0 && gy < S.H && gx >= 0 && gx < S.W;
        lv[i] = calib_level(planar[e], planar[np + e], t);
        if (in) rf[i] = inv_flat(planar[2 * np + e], flat_norm, status);
      }
      c += dc;
      r += dr;
      if (c >= mw) {
        c -= mw;
        ++r;
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int e = threadIdx.x + kThreads * i;
      if (e < np) ((float2*)s_mast)[e] = make_float2(lv[i], rf[i]);
    }
  } else {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = warp; r < mh; r += kThreads / 32) {
      const int gy = gy0 + r;
      const bool yin = gy >= 0 && gy < S.H;
      for (int c = lane; c < mw; c += 32) {
        const int gx = gx0 + c;
        float* dp = (float*)(s_mast + r * mw + c);
        const bool in = yin && gx >= 0 && gx < S.W;
        const float rf = in ? inv_flat(dp[2], flat_norm, status) : 0.0f;
        // fourth component: 1 for a pixel the bad-pixel mask marks
        const float mb =
            (in && S.mask && __ldg(S.mask + (int64_t)gy * S.mask_pitch + gx)) ? 1.0f : 0.0f;
        *(float2*)(dp + 2) = make_float2(rf, mb);
      }
    }
  }
  __syncthreads();
}

// The stencil over the lane's calibrated source rows v: the PY samples of
// the lane's output column (horizontal taps from the neighbouring lanes by
// shuffles, vertical taps from the lane's own rows).
template <int STENCIL, int SRC, int PY>
__device__ __forceinline__ void resample_rows(const FrameRec& F,
                                              const float (&v)[StageShape<SRC, STENCIL, PY>::rows],
                                              float (&a)[PY]) {
  using SS = StageShape<SRC, STENCIL, PY>;
  if (STENCIL == ST_NEAREST) {
#pragma unroll
    for (int q = 0; q < PY; ++q) a[q] = v[q];
  } else if (STENCIL == ST_BILINEAR) {
    const float2 w = *(const float2*)&F.fx;
    float hrow[SS::rows];
#pragma unroll
    for (int r = 0; r < SS::rows; ++r) {
      const float p1 = __shfl_down_sync(0xffffffffu, v[r], 1);
      hrow[r] = __fmaf_rn(w.x, __fsub_rn(p1, v[r]), v[r]);
    }
#pragma unroll
    for (int q = 0; q < PY; ++q) a[q] = __fmaf_rn(w.y, __fsub_rn(hrow[q + 1], hrow[q]), hrow[q]);
  } else if (STENCIL == ST_BSPLINE_V) {
    const float4 wy = *(const float4*)F.wy;
#pragma unroll
    for (int q = 0; q < PY; ++q) {
      float acc = wy.x * v[q];
      acc = __fmaf_rn(wy.y, v[q + 1], acc);
      acc = __fmaf_rn(wy.z, v[q + 2], acc);
      a[q] = __fmaf_rn(wy.w, v[q + 3], acc);
    }
  } else {  // ST_BSPLINE (coefficients) or ST_CUBIC (calibrated raw): 4x4 taps
    const float4 wx = *(const float4*)F.wx;
    const float4 wy = *(const float4*)F.wy;
    float hrow[SS::rows];
#pragma unroll
    for (int r = 0; r < SS::rows; ++r) {
      const float p1 = __shfl_down_sync(0xffffffffu, v[r], 1);
      const float p2 = __shfl_down_sync(0xffffffffu, v[r], 2);
      const float p3 = __shfl_down_sync(0xffffffffu, v[r], 3);
      float acc = wx.x * v[r];
      acc = __fmaf_rn(wx.y, p1, acc);
      acc = __fmaf_rn(wx.z, p2, acc);
      hrow[r] = __fmaf_rn(wx.w, p3, acc);
    }
#pragma unroll
    for (int q = 0; q < PY; ++q) {
      float acc = wy.x * hrow[q];
      acc = __fmaf_rn(wy.y, hrow[q + 1], acc);
      acc = __fmaf_rn(wy.z, hrow[q + 2], acc);
      a[q] = __fmaf_rn(wy.w, hrow[q + 3], acc);
    }
  }
}

// The lane's staged source rows of one frame of an interior tile (every
// pixel inside the frame, no mask): raw sources calibrated with the premerged
// window {bias + dark*t, rf} (PK = 1), coefficient sources as staged.
template <int STENCIL, int SRC, int PY, int PK>
__device__ __forceinline__ void load_rows_fast(const FrameRec& F, const uint8_t* st,
                                               const void* s_mast_w, int mrow, int lane,
                                               float (&v)[StageShape<SRC, STENCIL, PY>::rows]) {
  static_assert(SRC != SRC_RAW || PK == 1, "interior raw tiles read the premerged window");
  using SS = StageShape<SRC, STENCIL, PY>;
  const int2 g = *(const int2*)&F.off;  // off, mofs
  if (SRC == SRC_RAW) {
    const uint16_t* raw = (const uint16_t*)st + lane + g.x;
    const float2* mp = (const float2*)s_mast_w + g.y;
#pragma unroll
    for (int r = 0; r < SS::rows; ++r) {
      const float2 m = mp[r * mrow];
      v[r] = __fmul_rn(__fsub_rn(u16_to_float(raw[r * SS::elems]), m.x), m.y);
    }
  } else {
    const float* cf = (const float*)st + lane + g.x;
#pragma unroll
    for (int r = 0; r < SS::rows; ++r) v[r] = cf[r * SS::elems];
  }
}

// One frame of the warp's strip: calibrate the staged source rows, resample
// them to the strip's PY output rows, store the samples (+inf when invalid)
// and count the valid ones per row.
// MODE kFast: every sample of the tile valid, masters from the union window,
// no stack output (the interior of a set: no validity tests or counts);
// MODE kGeneral: validity per sample, masters and stack output decided per call.
// s_mast_w points at the warp's lane in the union window: float4 entries, or
// float2 entries when the window is premerged (PK = 1, or PK = 2 with pk set).
constexpr int kFast = 0, kGeneral = 1;

template <int STENCIL, int SRC, int PY, int MODE, int PK>
__device__ __forceinline__ void frame_step(const FrameRec& F, const uint8_t* st,
                                           const void* s_mast_w, int mrow, bool pk,
                                           const SetDesc& S, float flat_norm, uint32_t* status,
                                           int lane, int x, int tx0, int wy0, float* sk,
                                           int (&mq)[PY], float* stack_out, int k, int W, int H,
                                           int64_t out_pitch, bool stack_lane, bool norm) {
  using SS = StageShape<SRC, STENCIL, PY>;
  float v[SS::rows];
  float a[PY];
  if constexpr (MODE == kFast) {
    load_rows_fast<STENCIL, SRC, PY, PK>(F, st, s_mast_w, mrow, lane, v);
    resample_rows<STENCIL, SRC, PY>(F, v, a);
    if (norm) {
#pragma unroll
      for (int q = 0; q < PY; ++q) a[q] = __fmaf_rn(a[q], F.na, F.nz);
    }
#pragma unroll
    for (int q = 0; q < PY; ++q) sk[q * 32] = a[q];
    return;
  }
  const int4 g = *(const int4*)&F.off;      // off, mofs, vx0, vxw
  const float4 w = *(const float4*)&F.fx;   // fx, fy, t
  const int4 gy = *(const int4*)&F.vy0;     // vy0, vyw, ox, oy
  bool bad[SS::rows];  // bad source pixels (mask or saturation)
#pragma unroll
  for (int r = 0; r < SS::rows; ++r) bad[r] = false;
  const bool masked = S.masked;
  if (SRC == SRC_RAW) {
    const uint16_t* raw = (const uint16_t*)st + lane + g.x;
    if (mrow > 0 && (PK == 1 || (PK == 2 && pk))) {  // premerged window: never masked
      const float2* mp = (const float2*)s_mast_w + g.y;
#pragma unroll
      for (int r = 0; r < SS::rows; ++r) {
        const float2 m = mp[r * mrow];
        v[r] = __fmul_rn(__fsub_rn(u16_to_float(raw[r * SS::elems]), m.x), m.y);
      }
    } else if (mrow > 0) {
      const float4* mp = (const float4*)s_mast_w + g.y;
#pragma unroll
      for (int r = 0; r < SS::rows; ++r) {
        const float4 m = mp[r * mrow];
        const uint16_t q = raw[r * SS::elems];
        v[r] = calibrate_px(q, m.x, m.y, w.z, m.z);
        bad[r] = masked && (m.w != 0.0f || (float)q >= S.saturation);
      }
    } else {  // offsets too spread for a union window: masters from global memory
      const int gx = tx0 + gy.z + lane;
#pragma unroll
      for (int r = 0; r < SS::rows; ++r) {
        const int yy = wy0 + gy.w + r;
        float b = 0.0f, d = 0.0f, rf = 0.0f;
        bool mb = false;
        if (gx >= 0 && gx < S.W && yy >= 0 && yy < S.H) {
          const int64_t o = (int64_t)yy * S.master_pitch + gx;
          b = __ldg(S.bias + o);
          d = __ldg(S.dark + o);
          rf = inv_flat(__ldg(S.flat + o), flat_norm, status);
          mb = S.mask && __ldg(S.mask + (int64_t)yy * S.mask_pitch + gx);
        }
        const uint16_t q = raw[r * SS::elems];
        v[r] = calibrate_px(q, b, d, w.z, rf);
        bad[r] = masked && (mb || (float)q >= S.saturation);
      }
    }
  } else {
    const float* cf = (const float*)st + lane + g.x;
#pragma unroll
    for (int r = 0; r < SS::rows; ++r) v[r] = cf[r * SS::elems];
  }
  resample_rows<STENCIL, SRC, PY>(F, v, a);
  if (norm) {  // per-frame normalisation before the combine
#pragma unroll
    for (int q = 0; q < PY; ++q) a[q] = __fmaf_rn(a[q], F.na, F.nz);
  }
  const float kInf = __int_as_float(0x7f800000);
  const bool xv = in_range(x, g.z, g.w);
  // a sample is also invalid when a tap with non-zero weight is a bad pixel
  bool badq[PY];
#pragma unroll
  for (int q = 0; q < PY; ++q) badq[q] = false;
  if (SRC == SRC_RAW && masked) {
    if (STENCIL == ST_NEAREST) {
#pragma unroll
      for (int q = 0; q < PY; ++q) badq[q] = bad[q];
    } else if (STENCIL == ST_CUBIC) {
      // taps at lanes l .. l + 3 and rows q .. q + 3; with a zero fraction
      // only the tap at l + 1 (row q + 1) has non-zero weight
      const bool allx = (F.last_tap & 1) != 0, ally = (F.last_tap & 2) != 0;
      bool bh[SS::rows];
#pragma unroll
      for (int r = 0; r < SS::rows; ++r) {
        const int b1 = __shfl_down_sync(0xffffffffu, (int)bad[r], 1);
        const int b2 = __shfl_down_sync(0xffffffffu, (int)bad[r], 2);
        const int b3 = __shfl_down_sync(0xffffffffu, (int)bad[r], 3);
        bh[r] = allx ? (bad[r] | (b1 != 0) | (b2 != 0) | (b3 != 0)) : (b1 != 0);
      }
#pragma unroll
      for (int q = 0; q < PY; ++q)
        badq[q] = ally ? (bh[q] | bh[q + 1] | bh[q + 2] | bh[q + 3]) : bh[q + 1];
    } else {
      bool bh[SS::rows];
#pragma unroll
      for (int r = 0; r < SS::rows; ++r) {
        const int right = __shfl_down_sync(0xffffffffu, (int)bad[r], 1);
        bh[r] = bad[r] | ((w.x > 0.0f) & (right != 0));
      }
#pragma unroll
      for (int q = 0; q < PY; ++q) badq[q] = bh[q] | ((w.y > 0.0f) & bh[q + 1]);
    }
  }
  if (sk) {  // null for a stack-only set
#pragma unroll
    for (int q = 0; q < PY; ++q) {
      const bool ok = xv & in_range(wy0 + q, gy.x, gy.y) & !badq[q];
      sk[q * 32] = ok ? a[q] : kInf;
      mq[q] += ok ? 1 : 0;
    }
  }
  if (stack_out) {
#pragma unroll
    for (int q = 0; q < PY; ++q) {
      const int y = wy0 + q;
      const bool ok = xv & in_range(y, gy.x, gy.y) & !badq[q];
      if (stack_lane && y < H)
        stack_out[((int64_t)k * H + y) * out_pitch + x] = ok ? a[q] : __int_as_float(0x7fc00000);
    }
  }
}

// Two frames of an interior tile at once: both frames' rows are loaded before
// either is resampled and both results are stored last, so that the two
// dependency chains interleave.
template <int STENCIL, int SRC, int PY, int PK>
__device__ __forceinline__ void frame_pair_fast(const FrameRec& F0, const FrameRec& F1,
                                                const uint8_t* st0, const uint8_t* st1,
                                                const void* s_mast_w, int mrow, int lane,
                                                float* sk0, float* sk1, bool norm) {
  using SS = StageShape<SRC, STENCIL, PY>;
  float v0[SS::rows], v1[SS::rows];
  load_rows_fast<STENCIL, SRC, PY, PK>(F0, st0, s_mast_w, mrow, lane, v0);
  load_rows_fast<STENCIL, SRC, PY, PK>(F1, st1, s_mast_w, mrow, lane, v1);
  float a0[PY], a1[PY];
  resample_rows<STENCIL, SRC, PY>(F0, v0, a0);
  resample_rows<STENCIL, SRC, PY>(F1, v1, a1);
  if (norm) {
#pragma unroll
    for (int q = 0; q < PY; ++q) {
      a0[q] = __fmaf_rn(a0[q], F0.na, F0.nz);
      a1[q] = __fmaf_rn(a1[q], F1.na, F1.nz);
    }
  }
#pragma unroll
  for (int q = 0; q < PY; ++q) {
    sk0[q * 32] = a0[q];
    sk1[q * 32] = a1[q];
  }
}

template <int NMAX, int STENCIL, int SRC, int PY>
__device__ __forceinline__ void reduce_tile(const PlanView& P, int item, float* smem) {
  constexpr int kStages = stage_count(SRC, STENCIL, PY);
  constexpr int TH = 8 * PY;
  constexpr int TW = StencilShape<STENCIL>::tw;
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
  // the masters' window first (one cp.async group), so that its latency
  // overlaps the frame records and the first frames' staging
  const bool uwin = SRC == SRC_RAW && mwin_w > 0;
  const bool pk = uwin && (S.mflags & 2);  // premerged {bias + dark*t, rf} window
  if (uwin) issue_masters(S, tx0, ty0, s_mast, pk);
  cp_async_commit();
  int rec_fast = 1;
  for (int k = threadIdx.x; k < n; k += kThreads) {
    const FrameRec R = make_rec<SRC, STENCIL>(P.frames[S.frame0 + k], tx0, ty0, pitch, S.mox,
                                              S.moy, mwin_w, SS::rows + TH - PY, SS::elems,
                                     Hlim, Wlim, min(tx0 + TW, W) - 1, min(ty0 + TH, H) - 1);
    s_rec[k] = R;
    rec_fast &= (R.flags & 6) == 6 && (SRC != SRC_RAW || (R.flags & 1));
  }
  float flat_norm = 1.0f;
  if (SRC == SRC_RAW && S.flat_sum) flat_norm = (float)(*S.flat_sum / ((double)S.W * S.H));
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
    LC.has[it] = c < SS::rows * SS::chunks;
    LC.soff[it] = LC.has[it] ? c * 16 : 0;
    LC.goff[it] = ((int64_t)LC.drow[it] * pitch + LC.dcol[it]) * esz;
  }
  // the tile's class: interior tiles (every frame aligned, staged without
  // bounds checks and valid at every pixel) take the branch-free loop
  const bool tile_fast = __syncthreads_and(rec_fast) && (SRC != SRC_RAW || mwin_w > 0) &&
                         !stack_out && !S.masked && !S.stack_only;

  const FrameRec* frames = s_rec;
  const bool norm = h.frame_norm != 0;
  // interior tiles of raw sources with a premerged master window take the
  // frames two at a time; those of several exposure times take the general
  // loop
  constexpr bool kPairs = pair_frames(SRC, PY) && kStages % 2 == 0 && kStages >= 4;
  const bool pairs = kPairs && tile_fast && pk;
  // prologue: frames 0 .. kStages-2 in flight, one group each (single
  // steps), or frames 0 .. kStages-3 in groups of two (pairs); then wait for
  // the masters' group, the oldest, alone and turn it into the window
  if (pairs) {
#pragma unroll
    for (int j = 0; j < (kStages - 2) / 2; ++j) {
      if (2 * j < n)
        issue_stage_inside<SRC, kIt>(frames[2 * j], LC, s_stage + (2 * j) * SS::bytes);
      if (2 * j + 1 < n)
        issue_stage_inside<SRC, kIt>(frames[2 * j + 1], LC, s_stage + (2 * j + 1) * SS::bytes);
      cp_async_commit();
    }
    cp_async_wait<(kStages - 2) / 2>();
  } else {
#pragma unroll
    for (int k = 0; k < kStages - 1; ++k) {
      if (k < n)
        issue_stage<SRC, STENCIL, PY>(frames[k], LC, Hlim, Wlim, pitch, s_stage + k * SS::bytes,
                                      lane, warp * PY);
      cp_async_commit();
    }
    cp_async_wait<kStages - 1>();
  }
  __syncthreads();
  if (uwin) finish_masters(S, tx0, ty0, flat_norm, s_mast, pk, frames[0].t, h.status);
  // the warp's lane in the union window: float2 entries when premerged, else
  // float4 entries
  const void* s_mast_w = pk ? (const void*)((const float2*)s_mast + warp * PY * mwin_w + lane)
                            : (const void*)(s_mast + warp * PY * mwin_w + lane);
  const bool stack_lane = lane < TW && x < W;
  int mq[PY];
#pragma unroll
  for (int q = 0; q < PY; ++q) mq[q] = 0;
  // a stack-only set (a chunk of a set deeper than the register buckets) keeps
  // no samples: its group reserves no shared memory for them
  float* sk = S.stack_only ? nullptr : s_samples + (size_t)warp * PY * 32 + lane;
  // single frames in groups of kStages (slots constant in the unrolled groups)
  auto step = [&](auto mode, auto packed, int k, int u, bool issue_next) {
    constexpr int MODE = decltype(mode)::value;
    constexpr int PK = decltype(packed)::value;
    cp_async_wait<kStages - 2>();
    __syncwarp();
    if (issue_next) {
      uint8_t* dst = s_stage + ((u + kStages - 1) % kStages) * SS::bytes;
      if (MODE == kFast)
        issue_stage_inside<SRC, kIt>(frames[k + kStages - 1], LC, dst);
      else
        issue_stage<SRC, STENCIL, PY>(frames[k + kStages - 1], LC, Hlim, Wlim, pitch, dst, lane,
                                      warp * PY);
    }
    cp_async_commit();
    frame_step<STENCIL, SRC, PY, MODE, PK>(frames[k], s_stage + u * SS::bytes, s_mast_w, mwin_w,
                                           pk, S, flat_norm, h.status, lane, x, tx0, wy0,
                                           sk ? sk + (size_t)k * TH * 32 : nullptr, mq,
                                           stack_out, k, W, H, out_pitch, stack_lane, norm);
  };
  auto frame_loop = [&](auto mode, auto packed) {
    int k0 = 0;
    // groups whose frames and whose successors' copies all exist: no tests
    for (; k0 + 2 * kStages - 1 <= n; k0 += kStages) {
#pragma unroll
      for (int u = 0; u < kStages; ++u) step(mode, packed, k0 + u, u, true);
    }
    for (; k0 < n; k0 += kStages) {
#pragma unroll 1
      for (int u = 0; u < kStages; ++u)
        if (k0 + u < n) step(mode, packed, k0 + u, u, k0 + u + kStages - 1 < n);
    }
  };
  // frame pairs (k, k + 1) in stage slots (u, u + 1): wait for the pair,
  // issue frames k + kStages - 2 and k + kStages - 1 into the slots of the
  // previous pair, then compute the pair (or the last, odd frame alone)
  auto pair_step = [&](auto packed, int k, int u, bool full) {
    constexpr int PK = decltype(packed)::value;
    cp_async_wait<(kStages - 4) / 2>();
    __syncwarp();
    const int ka = k + kStages - 2, kb = k + kStages - 1;
    if (full || ka < n)
      issue_stage_inside<SRC, kIt>(frames[ka], LC,
                                   s_stage + ((u + kStages - 2) % kStages) * SS::bytes);
    if (full || kb < n)
      issue_stage_inside<SRC, kIt>(frames[kb], LC,
                                   s_stage + ((u + kStages - 1) % kStages) * SS::bytes);
    cp_async_commit();
    float* sk0 = sk + (size_t)k * TH * 32;
    if (full || k + 1 < n) {
      frame_pair_fast<STENCIL, SRC, PY, PK>(frames[k], frames[k + 1], s_stage + u * SS::bytes,
                                            s_stage + (u + 1) * SS::bytes, s_mast_w, mwin_w,
                                            lane, sk0, sk0 + TH * 32, norm);
    } else {
      frame_step<STENCIL, SRC, PY, kFast, PK>(frames[k], s_stage + u * SS::bytes, s_mast_w,
                                              mwin_w, pk, S, flat_norm, h.status, lane, x, tx0,
                                              wy0, sk0, mq, nullptr, k, W, H, out_pitch,
                                              stack_lane, norm);
    }
  };
  auto pair_loop = [&](auto packed) {
    int k0 = 0;
    // groups of kStages frames whose successors' copies all exist: no tests
    for (; k0 + 2 * kStages - 2 <= n; k0 += kStages) {
#pragma unroll
      for (int u = 0; u < kStages; u += 2) pair_step(packed, k0 + u, u, true);
    }
    for (; k0 < n; k0 += kStages) {
#pragma unroll 1
      for (int u = 0; u < kStages; u += 2)
        if (k0 + u < n) pair_step(packed, k0 + u, u, false);
    }
  };
  using I1 = std::integral_constant<int, 1>;
  using I2 = std::integral_constant<int, 2>;
  // interior tiles of raw sources need the premerged window (frames of
  // several exposure times take the general loop); coefficient sources read
  // no masters
  const bool fast = tile_fast && (pk || SRC != SRC_RAW);
  if constexpr (kPairs) {
    if (pairs)
      pair_loop(I1{});
    else
      frame_loop(std::integral_constant<int, kGeneral>{}, I2{});
  } else {
    if (fast)
      frame_loop(std::integral_constant<int, kFast>{}, I1{});
    else
      frame_loop(std::integral_constant<int, kGeneral>{}, I2{});
  }
  cp_async_wait<0>();
  __syncwarp();

  const ClipArgs ca{h.kappa_lo, h.kappa_hi, h.max_iter, h.center, h.ddof};
  float* const mean_out = S.mean_out;
  float* const median_out = S.median_out;
  uint16_t* const nkept_out = S.nkept_out;
  constexpr int kSure = bucket_below(NMAX);  // every set of this bucket has more frames
  const float kInf = __int_as_float(0x7f800000);
  if (!S.stack_only && lane < TW && x < W) {
#pragma unroll 1
    for (int q = 0; q < PY; ++q) {
      const int y = wy0 + q;
      if (y >= H) break;
      const float* sp = s_samples + (size_t)(warp * PY + q) * 32 + lane;
      float s[NMAX];
#pragma unroll
      for (int j = 0; j < NMAX; ++j)
        s[j] = (j < kSure || j < n) ? sp[(size_t)j * TH * 32] : kInf;
      sort_network<NMAX>(s);
      int m = mq[0];
#pragma unroll
      for (int qq = 1; qq < PY; ++qq) m = (q == qq) ? mq[qq] : m;
      if (tile_fast) m = n;
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

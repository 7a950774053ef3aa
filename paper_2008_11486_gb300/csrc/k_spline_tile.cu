// k_spline_tile.cu -- the cubic-spline reduction of one output tile, from the
// row-pass coefficients of its frames to the combined pixels, in one kernel.
//
// Sec. 2.1 aligns the frames by bicubic-spline interpolation and co-adds them
// by a sigma-clipped mean; Sec. 3.2.1 solves one tridiagonal system per row
// and per column for the spline.  The row systems are solved by the row pass
// (k_spline.cu), which leaves each frame's rows filtered along x ("row-pass
// coefficients", FP32 on the source grid).  This kernel does the rest for a
// tile of 29 output columns x TH output rows:
//   1. per frame, lane l solves the column system of the source column that
//      the frame's first horizontal tap of output column tx0 + l falls on, by
//      the causal and anti-causal recursions (pole z1 = sqrt(3) - 2), each
//      started 16 rows outside the rows it keeps (|z1|^16 = 7e-10) and reading
//      the mirror-extended column at the frame's edges;
//   2. the 4 horizontal B-spline taps come from lanes l .. l + 3 by shuffles,
//      the 4 vertical taps from the lane's own rows, in the 4x4 evaluation's
//      order, giving the frame's sample of each output pixel of the column;
//   3. invalid samples (source position outside the frame, or a tap with
//      non-zero weight on a bad pixel) become +inf, and the samples go to
//      shared memory;
//   4. after the last frame each lane combines its pixels (combine.cuh).
// The 8 warps take the frames round-robin.  Only the row-pass coefficients
// cross HBM (or, when the launch sequence keeps them resident, L2) between
// the two passes: the column coefficients and the filtered rows stay on chip.
#include "reduce_kernels.cuh"
#include "spline.h"
#include "wide.cuh"

namespace irp {

namespace {

constexpr int kTileWarm = 16;  // warm-up rows of each column recursion

// Tile height by register bucket: the samples of a tile ([n][TH][32] floats)
// stay within 64 KB of shared memory.
template <int NMAX>
struct SplineTileShape {
  static constexpr int th = NMAX <= 16 ? 32 : (NMAX <= 32 ? 16 : 8);
  // resident CTAs per SM the register allocation must allow (at most 85
  // registers per thread for three)
  static constexpr int min_blocks = NMAX <= 16 ? 3 : 2;
};

__device__ __forceinline__ void grid_dependency_wait() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

}  // namespace

// What a task needs of one frame, staged in shared memory once per tile (96 bytes).
struct TileFrame {
  const float* crow;
  const uint32_t* bad;
  float wx[4], wy[4];
  int ox, oy, vx0, vx1;
  int vy0, vy1, last_tap, pad0;
  float na, nz;  // per-frame normalisation: sample = fma(sample, na, nz)
  int pad1[2];
};
static_assert(sizeof(TileFrame) == 96, "TileFrame layout");

// Stages the set's frame fields for a tile of kSplineTileCols x th output
// rows from (tx0, ty0) in shared memory (threads stride the frames); returns
// whether every frame this thread staged is valid at every pixel of the tile.
__device__ __forceinline__ int fill_tile_frames(const PlanView& P, const SetDesc& S,
                                                TileFrame* s_frames, int tx0, int ty0, int th) {
  int all_valid = 1;
  const int W = S.W, H = S.H;
  for (int k = threadIdx.x; k < S.n; k += kThreads) {
    const FrameDesc& F = P.frames[S.frame0 + k];
    TileFrame T;
    T.crow = F.crow;
    T.bad = F.bad;
    for (int i = 0; i < 4; ++i) {
      T.wx[i] = F.wx[i];
      T.wy[i] = F.wy[i];
    }
    T.na = F.norm ? F.norm->na : 1.0f;
    T.nz = F.norm ? F.norm->nz : 0.0f;
    T.pad1[0] = T.pad1[1] = 0;
    T.ox = F.ox;
    T.oy = F.oy;
    T.vx0 = F.vx0;
    T.vx1 = F.vx1;
    T.vy0 = F.vy0;
    T.vy1 = F.vy1;
    T.last_tap = F.last_tap;
    T.pad0 = 0;
    s_frames[k] = T;
    all_valid &= F.vx0 <= tx0 && F.vx1 >= min(tx0 + kSplineTileCols, W) - 1 && F.vy0 <= ty0 &&
                 F.vy1 >= min(ty0 + th, H) - 1;
  }
  return all_valid;
}

// One task of a tile kernel: frame k's samples of the TR output rows from ry0
// on, in the column of lane l (output column x): the column recursions of the
// row-pass coefficients the frame's first horizontal tap of x falls on (16
// warm-up rows at either end), the 4 horizontal taps by shuffles, the bad-pixel
// footprint and the 4 vertical taps.  emit(q, v) receives the sample of row
// ry0 + q, +inf when invalid; the caller's aligned stack (debug output) gets
// NaN there.
template <int TR, typename Emit>
__device__ __forceinline__ void spline_task(const SetDesc& S, const TileFrame& F, int k, int ry0,
                                            int x, int lane, bool masked, bool norm, Emit emit) {
  constexpr int NC = TR + 3;                 // coefficient rows: the vertical taps of TR rows
  constexpr int NR = NC + 2 * kTileWarm;     // rows each lane reads per task
  const int W = S.W, H = S.H;
  const int64_t cpitch = S.crow_pitch;
  const float kInf = __int_as_float(0x7f800000);
  const int cx = mirror_index(x + F.ox, W);
  const float* col = F.crow + cx;
  const int r0 = ry0 + F.oy - kTileWarm;
  float v[NR];
  if (r0 >= 0 && r0 + NR <= H) {
    const float* p = col + (int64_t)r0 * cpitch;
#pragma unroll
    for (int j = 0; j < NR; ++j) v[j] = __ldg(p + (int64_t)j * cpitch);
  } else {
#pragma unroll
    for (int j = 0; j < NR; ++j) v[j] = __ldg(col + (int64_t)mirror_index(r0 + j, H) * cpitch);
  }
  // causal recursion from zero through the upper warm-up rows; c keeps y+
  float c[NC];
  {
    float a = 0.0f;
#pragma unroll
    for (int j = 0; j < kTileWarm; ++j) a = __fmaf_rn(kZ1, a, v[j]);
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      a = __fmaf_rn(kZ1, a, v[kTileWarm + j]);
      c[j] = a;
    }
  }
  // anti-causal recursion from zero through the lower warm-up rows, and the
  // coefficients c = sqrt(3) (y+ + y- - v)
  {
    float b = 0.0f;
#pragma unroll
    for (int j = NR - 1; j >= kTileWarm + NC; --j) b = __fmaf_rn(kZ1, b, v[j]);
#pragma unroll
    for (int j = NC - 1; j >= 0; --j) {
      b = __fmaf_rn(kZ1, b, v[kTileWarm + j]);
      c[j] = __fmul_rn(kSqrt3, __fsub_rn(__fadd_rn(c[j], b), v[kTileWarm + j]));
    }
  }
  // horizontal taps from lanes l .. l + 3 (left to right), in place
  const float4 wx = *reinterpret_cast<const float4*>(F.wx);
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    const float c1 = __shfl_down_sync(0xffffffffu, c[j], 1);
    const float c2 = __shfl_down_sync(0xffffffffu, c[j], 2);
    const float c3 = __shfl_down_sync(0xffffffffu, c[j], 3);
    float hh = wx.x * c[j];
    hh = __fmaf_rn(wx.y, c1, hh);
    hh = __fmaf_rn(wx.z, c2, hh);
    c[j] = __fmaf_rn(wx.w, c3, hh);
  }
  // bad-pixel footprint: bit j of `badrows` marks coefficient row j of this
  // lane's source column bad; a sample is invalid when any tap with non-zero
  // weight (columns l .. l + 3, rows q .. q + 3) is bad
  uint32_t badq = 0;
  if (masked) {
    const uint32_t* bits = F.bad + (cx >> 5);
    const int sh = cx & 31;
    const int64_t bp = S.bad_pitch;
    const int rb = ry0 + F.oy;
    uint32_t badrows = 0;
#pragma unroll
    for (int j = 0; j < NC; ++j)
      badrows |= ((__ldg(bits + (int64_t)mirror_index(rb + j, H) * bp) >> sh) & 1u) << j;
    // with the fraction f in [0, 1) the first three taps of an axis always
    // have non-zero weight, the fourth, beta3(2 - f), unless f = 0
    uint32_t cols = badrows | __shfl_down_sync(0xffffffffu, badrows, 1) |
                    __shfl_down_sync(0xffffffffu, badrows, 2);
    const uint32_t c3 = __shfl_down_sync(0xffffffffu, badrows, 3);
    if (F.last_tap & 1) cols |= c3;
    badq = cols | (cols >> 1) | (cols >> 2);
    if (F.last_tap & 2) badq |= cols >> 3;
  }
  const float4 wy = *reinterpret_cast<const float4*>(F.wy);
  const bool xv = F.vx1 >= F.vx0 && in_range(x, F.vx0, F.vx1 - F.vx0);
  // the caller's aligned stack (debug output): NaN for invalid samples
  float* const st = (S.stack_out && lane < kSplineTileCols && x < W)
                        ? S.stack_out + (int64_t)k * H * S.out_pitch + x : nullptr;
#pragma unroll
  for (int q = 0; q < TR; ++q) {
    float acc = wy.x * c[q];
    acc = __fmaf_rn(wy.y, c[q + 1], acc);
    acc = __fmaf_rn(wy.z, c[q + 2], acc);
    acc = __fmaf_rn(wy.w, c[q + 3], acc);
    if (norm) acc = __fmaf_rn(acc, F.na, F.nz);  // per-frame normalisation
    const int y = ry0 + q;
    const bool ok = xv && y >= F.vy0 && y <= F.vy1 && !((badq >> q) & 1u);
    emit(q, ok ? acc : kInf);
    if (st && y < H) st[(int64_t)y * S.out_pitch] = ok ? acc : __int_as_float(0x7fc00000);
  }
}

template <int NMAX>
__global__ void __launch_bounds__(kThreads, SplineTileShape<NMAX>::min_blocks)
    k_spline_tile(const __grid_constant__ InlinePlan inl, const void* plan_dev, int item0) {
  constexpr int TH = SplineTileShape<NMAX>::th;
  constexpr int TR = TH < 16 ? TH : 16;      // output rows per task (frame, row block)
  constexpr int NB = TH / TR;                // row blocks per tile
  constexpr int RPW = TH / 8;                // output rows each warp combines
  extern __shared__ float4 smem4[];
  float* s_samples = reinterpret_cast<float*>(smem4);  // [n][TH][32]
  TileFrame* s_frames = reinterpret_cast<TileFrame*>(s_samples + (size_t)NMAX * TH * 32);
  grid_dependency_wait();                    // the row pass (launched before) is complete
  const PlanView P = make_view(inl, plan_dev);
  const PlanHeader& h = *P.h;
  const int item = item0 + (int)blockIdx.x;
  if (item >= h.nitems) return;
  const SetDesc& S = P.sets[find_set(P.sets, h.nsets, item)];
  const int tile = item - S.tile0;
  const int tx0 = (tile % S.tiles_x) * kSplineTileCols;
  const int ty0 = (tile / S.tiles_x) * TH;
  const int W = S.W, H = S.H, n = S.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int x = tx0 + lane;
  const float kInf = __int_as_float(0x7f800000);
  const bool masked = S.masked != 0;
  // the frames' fields, once per tile; and whether every frame is valid at
  // every pixel of the tile (the combine then knows the count)
  const int all_valid = fill_tile_frames(P, S, s_frames, tx0, ty0, TH);
  const bool tile_valid = __syncthreads_and(all_valid) && !masked;
  const bool norm = h.frame_norm != 0;

  // tasks (frame, block of TR output rows), round-robin over the warps
#pragma unroll 1
  for (int task = warp; task < n * NB; task += kThreads / 32) {
    const int k = NB == 1 ? task : task / NB;
    const int ry0 = ty0 + (task - k * NB) * TR;  // first output row of the task
    float* sk = s_samples + ((size_t)k * TH + (ry0 - ty0)) * 32 + lane;
    spline_task<TR>(S, s_frames[k], k, ry0, x, lane, masked, norm,
                    [&](int q, float v) { sk[q * 32] = v; });
  }
  __syncthreads();

  const ClipArgs ca{h.kappa_lo, h.kappa_hi, h.max_iter, h.center, h.ddof};
  constexpr int kSure = bucket_below(NMAX);  // every set of this bucket has more frames
  if (lane < kSplineTileCols && x < W) {
#pragma unroll 1
    for (int qq = 0; qq < RPW; ++qq) {
      const int q = warp * RPW + qq;
      const int y = ty0 + q;
      if (y >= H) break;
      const float* sp = s_samples + (size_t)q * 32 + lane;
      float s[NMAX];
      int m = 0;
#pragma unroll
      for (int j = 0; j < NMAX; ++j) {
        s[j] = (j < kSure || j < n) ? sp[(size_t)j * TH * 32] : kInf;
        m += (s[j] != kInf) ? 1 : 0;
      }
      if (tile_valid) m = n;
      sort_network<NMAX>(s);
      const CombineOut o = combine_sorted<NMAX>(s, m, ca);
      const int64_t oi = (int64_t)y * S.out_pitch + x;
      if (S.mean_out) S.mean_out[oi] = o.mean;
      if (S.median_out) S.median_out[oi] = o.median;
      if (S.nkept_out) S.nkept_out[oi] = (uint16_t)o.kept;
    }
  }
}

// ---------------------------------------------------------------------------
// Sets of more frames than the register buckets hold (IRP_MAX_FRAMES < n <=
// kWideTileMax; the paper's bands hold 180): the same tasks, with the samples
// kept per output pixel in shared memory -- pixel p = q * 32 + l (row q, lane
// l) holds sample k at p * ps + k + k / 32, ps = wide_tile_stride(n) odd, so
// that both the tasks' stores (one frame, 32 pixels) and a group's loads
// (samples t J .. t J + J - 1 in lane t) fall on distinct banks -- and a
// group of G lanes combines each pixel (wide.cuh: a bitonic sort of G J
// values across the group, then the clip passes on the sorted run).  The
// frame table comes first in shared memory, then the samples.
// ---------------------------------------------------------------------------
template <int G, int TH>
__global__ void __launch_bounds__(kThreads, TH <= 4 ? 2 : 1)
    k_spline_tile_wide(const __grid_constant__ InlinePlan inl, const void* plan_dev, int item0) {
  constexpr int J = 32;
  constexpr int NPW = 32 / G;  // pixels a warp combines at a time
  static_assert((TH * 32) % (NPW * (kThreads / 32)) == 0, "whole rounds of pixels");
  extern __shared__ float4 smem4[];
  grid_dependency_wait();  // the row pass (launched before) is complete
  const PlanView P = make_view(inl, plan_dev);
  const PlanHeader& h = *P.h;
  const int item = item0 + (int)blockIdx.x;
  if (item >= h.nitems) return;
  const SetDesc& S = P.sets[find_set(P.sets, h.nsets, item)];
  const int tile = item - S.tile0;
  const int tx0 = (tile % S.tiles_x) * kSplineTileCols;
  const int ty0 = (tile / S.tiles_x) * TH;
  const int W = S.W, H = S.H, n = S.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int x = tx0 + lane;
  const bool masked = S.masked != 0;
  const float kInf = __int_as_float(0x7f800000);
  TileFrame* s_frames = reinterpret_cast<TileFrame*>(smem4);
  float* s_samples = reinterpret_cast<float*>(s_frames + n);  // 96 n bytes: 16-byte aligned
  const int ps = wide_tile_stride(n);
  fill_tile_frames(P, S, s_frames, tx0, ty0, TH);
  __syncthreads();
  const bool norm = h.frame_norm != 0;
  // tasks: one frame's TH rows each, round-robin over the warps
#pragma unroll 1
  for (int k = warp; k < n; k += kThreads / 32) {
    float* sk = s_samples + (size_t)lane * ps + k + (k >> 5);
    spline_task<TH>(S, s_frames[k], k, ty0, x, lane, masked, norm,
                    [&](int q, float v) { sk[(size_t)q * 32 * ps] = v; });
  }
  __syncthreads();
  const ClipArgs ca{h.kappa_lo, h.kappa_hi, h.max_iter, h.center, h.ddof};
  const int g = lane / G, tg = lane % G;  // the lane's group and its index in it
#pragma unroll 1
  for (int base = warp * NPW; base < TH * 32; base += (kThreads / 32) * NPW) {
    const int p = base + g;
    const int q = p >> 5, l = p & 31;
    const int px = tx0 + l, py = ty0 + q;
    const bool live = l < kSplineTileCols && px < W && py < H;
    float* const col = s_samples + (size_t)p * ps;  // this pixel's samples
    float v[J];
    int cnt = 0;
#pragma unroll
    for (int i = 0; i < J; ++i) {
      const int e = tg * J + i;
      v[i] = (live && e < n) ? col[e + e / J] : kInf;
      cnt += v[i] < kInf ? 1 : 0;
    }
    const int m = group_sum_i<G>(cnt);
    group_bitonic_sort<G, J>(v, tg);
    // the sorted run replaces the pixel's samples (only the first n are
    // stored; the order statistics read below index the valid run only)
    __syncwarp();
#pragma unroll
    for (int i = 0; i < J; ++i) {
      const int e = tg * J + i;
      if (live && e < n) col[e + e / J] = v[i];
    }
    __syncwarp();
    const WideOut o = group_combine<G, J>(v, col, m, ca, tg);
    if (live && tg == 0) {
      const int64_t oi = (int64_t)py * S.out_pitch + px;
      if (S.mean_out) S.mean_out[oi] = o.mean;
      if (S.median_out) S.median_out[oi] = o.median;
      if (S.nkept_out) S.nkept_out[oi] = (uint16_t)o.kept;
    }
  }
}

// Shared memory of the wide tile kernel: the frame table, then TH x 32 pixels
// of ps samples.
static size_t wide_tile_smem(int th, int max_n) {
  return (size_t)max_n * sizeof(TileFrame) + (size_t)th * 32 * wide_tile_stride(max_n) * sizeof(float);
}

int spline_tile_rows(int bucket, int max_n) {
  if (bucket > IRP_MAX_FRAMES)  // the wide kernel: 8 rows when they fit, else 4
    return wide_tile_smem(8, max_n) <= kWideTileSmem ? 8 : 4;
  return bucket <= 16 ? 32 : (bucket <= 32 ? 16 : 8);
}

size_t spline_tile_smem_bytes(int bucket, int max_n) {
  if (bucket > IRP_MAX_FRAMES) return wide_tile_smem(spline_tile_rows(bucket, max_n), max_n);
  // samples [bucket][TH][32] (the kernel lays out the frame table after the
  // bucket's samples), then the frame table
  return (size_t)bucket * spline_tile_rows(bucket, max_n) * 32 * sizeof(float) +
         (size_t)bucket * sizeof(TileFrame);
}

namespace {

template <typename Fn>
cudaError_t launch_tile_fn(Fn fn, size_t& granted, const InlinePlan* inl, const void* plan_dev,
                           int item0, int grid, size_t smem, cudaStream_t s, bool pdl) {
  cudaError_t e = ensure_smem(fn, smem, granted);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, fn, *inl, plan_dev, item0);
}

template <int NMAX>
cudaError_t launch_tile_bucket(const InlinePlan* inl, const void* plan_dev, int item0, int grid,
                               size_t smem, cudaStream_t s, bool pdl) {
  static size_t granted = 0;
  return launch_tile_fn(k_spline_tile<NMAX>, granted, inl, plan_dev, item0, grid, smem, s, pdl);
}

template <int G, int TH>
cudaError_t launch_tile_wide(const InlinePlan* inl, const void* plan_dev, int item0, int grid,
                             size_t smem, cudaStream_t s, bool pdl) {
  static size_t granted = 0;
  return launch_tile_fn(k_spline_tile_wide<G, TH>, granted, inl, plan_dev, item0, grid, smem, s,
                        pdl);
}

}  // namespace

cudaError_t launch_spline_tile(int bucket, int th, const InlinePlan* inl, const void* plan_dev,
                               int item0, int grid, size_t smem, cudaStream_t s, bool pdl) {
  if (bucket > IRP_MAX_FRAMES) {
    const bool g4 = wide_tile_g(bucket) == 4;
    if (th == 8)
      return g4 ? launch_tile_wide<4, 8>(inl, plan_dev, item0, grid, smem, s, pdl)
                : launch_tile_wide<8, 8>(inl, plan_dev, item0, grid, smem, s, pdl);
    if (th == 4 && !g4) return launch_tile_wide<8, 4>(inl, plan_dev, item0, grid, smem, s, pdl);
    return cudaErrorInvalidValue;
  }
  switch (bucket) {
#define IRP_TILE_CASE(B) \
  case B: return launch_tile_bucket<B>(inl, plan_dev, item0, grid, smem, s, pdl);
    IRP_FOR_BUCKETS(IRP_TILE_CASE)
#undef IRP_TILE_CASE
  }
  return cudaErrorInvalidValue;
}

}  // namespace irp

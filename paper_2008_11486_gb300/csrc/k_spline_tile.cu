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

namespace irp {

namespace {

constexpr int kTileWarm = 16;  // warm-up rows of each column recursion

// Tile height by register bucket: the samples of a tile ([n][TH][32] floats)
// stay within 64 KB of shared memory.
template <int NMAX>
struct SplineTileShape {
  static constexpr int th = NMAX <= 16 ? 32 : (NMAX <= 32 ? 16 : 8);
};

__device__ __forceinline__ void grid_dependency_wait() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

}  // namespace

template <int NMAX>
__global__ void __launch_bounds__(kThreads, 2)
    k_spline_tile(const __grid_constant__ InlinePlan inl, const void* plan_dev, int item0) {
  constexpr int TH = SplineTileShape<NMAX>::th;
  constexpr int NC = TH + 3;                 // coefficient rows: the vertical taps of TH rows
  constexpr int NR = NC + 2 * kTileWarm;     // rows each lane reads per frame
  constexpr int RPW = TH / 8;                // output rows each warp combines
  extern __shared__ float4 smem4[];
  float* s_samples = reinterpret_cast<float*>(smem4);  // [n][TH][32]
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
  const int64_t cpitch = S.crow_pitch;
  const int x = tx0 + lane;
  const float kInf = __int_as_float(0x7f800000);
  const bool masked = S.masked != 0;
  // every frame valid at every pixel of the tile: the combine knows the count
  int all_valid = 1;
  for (int k = threadIdx.x; k < n; k += kThreads) {
    const FrameDesc& F = P.frames[S.frame0 + k];
    all_valid &= F.vx0 <= tx0 && F.vx1 >= min(tx0 + kSplineTileCols, W) - 1 && F.vy0 <= ty0 &&
                 F.vy1 >= min(ty0 + TH, H) - 1;
  }
  const bool tile_valid = __syncthreads_and(all_valid) && !masked;

  for (int k = warp; k < n; k += kThreads / 32) {
    const FrameDesc& F = P.frames[S.frame0 + k];
    const int cx = mirror_index(x + F.ox, W);
    const float* col = F.crow + cx;
    const int r0 = ty0 + F.oy - kTileWarm;
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
    const float wx0 = F.wx[0], wx1 = F.wx[1], wx2 = F.wx[2], wx3 = F.wx[3];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      const float c1 = __shfl_down_sync(0xffffffffu, c[j], 1);
      const float c2 = __shfl_down_sync(0xffffffffu, c[j], 2);
      const float c3 = __shfl_down_sync(0xffffffffu, c[j], 3);
      float hh = wx0 * c[j];
      hh = __fmaf_rn(wx1, c1, hh);
      hh = __fmaf_rn(wx2, c2, hh);
      c[j] = __fmaf_rn(wx3, c3, hh);
    }
    // bad-pixel footprint: bit j of `badrows` marks coefficient row j of this
    // lane's source column bad; a sample is invalid when any tap with non-zero
    // weight (columns l .. l + 3, rows q .. q + 3) is bad
    uint64_t badq = 0;
    if (masked) {
      const uint32_t* bits = F.bad + (cx >> 5);
      const int sh = cx & 31;
      const int64_t bp = S.bad_pitch;
      const int rb = ty0 + F.oy;
      uint64_t badrows = 0;
#pragma unroll
      for (int j = 0; j < NC; ++j)
        badrows |= (uint64_t)((__ldg(bits + (int64_t)mirror_index(rb + j, H) * bp) >> sh) & 1u)
                   << j;
      // with the fraction f in [0, 1) the first three taps of an axis always
      // have non-zero weight, the fourth, beta3(2 - f), unless f = 0
      uint64_t cols = badrows | __shfl_down_sync(0xffffffffu, badrows, 1) |
                      __shfl_down_sync(0xffffffffu, badrows, 2);
      const uint64_t c3 = __shfl_down_sync(0xffffffffu, badrows, 3);
      if (F.last_tap & 1) cols |= c3;
      badq = cols | (cols >> 1) | (cols >> 2);
      if (F.last_tap & 2) badq |= cols >> 3;
    }
    const float wy0 = F.wy[0], wy1 = F.wy[1], wy2 = F.wy[2], wy3 = F.wy[3];
    const bool xv = in_range(x, F.vx0, F.vx1 - F.vx0) && F.vx1 >= F.vx0;
    float* sk = s_samples + (size_t)k * TH * 32 + lane;
    // the caller's aligned stack (debug output): NaN for invalid samples
    float* const st = (S.stack_out && lane < kSplineTileCols && x < W)
                          ? S.stack_out + (int64_t)k * H * S.out_pitch + x : nullptr;
#pragma unroll
    for (int q = 0; q < TH; ++q) {
      float acc = wy0 * c[q];
      acc = __fmaf_rn(wy1, c[q + 1], acc);
      acc = __fmaf_rn(wy2, c[q + 2], acc);
      acc = __fmaf_rn(wy3, c[q + 3], acc);
      const int y = ty0 + q;
      const bool ok = xv && y >= F.vy0 && y <= F.vy1 && !((badq >> q) & 1u);
      sk[q * 32] = ok ? acc : kInf;
      if (st && y < H) st[(int64_t)y * S.out_pitch] = ok ? acc : __int_as_float(0x7fc00000);
    }
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

size_t spline_tile_smem_bytes(int bucket, int max_n) {
  return (size_t)max_n * spline_tile_rows(bucket) * 32 * sizeof(float);
}

int spline_tile_rows(int bucket) { return bucket <= 16 ? 32 : (bucket <= 32 ? 16 : 8); }

namespace {

template <int NMAX>
cudaError_t launch_tile_bucket(const InlinePlan* inl, const void* plan_dev, int item0, int grid,
                               size_t smem, cudaStream_t s, bool pdl) {
  static size_t granted = 0;
  auto fn = k_spline_tile<NMAX>;
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

}  // namespace

cudaError_t launch_spline_tile(int bucket, const InlinePlan* inl, const void* plan_dev, int item0,
                               int grid, size_t smem, cudaStream_t s, bool pdl) {
  switch (bucket) {
#define IRP_TILE_CASE(B) \
  case B: return launch_tile_bucket<B>(inl, plan_dev, item0, grid, smem, s, pdl);
    IRP_FOR_BUCKETS(IRP_TILE_CASE)
#undef IRP_TILE_CASE
  }
  return cudaErrorInvalidValue;
}

}  // namespace irp

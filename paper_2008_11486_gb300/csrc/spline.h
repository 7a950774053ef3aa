// spline.h -- launchers of the row and column spline-coefficient passes.
#pragma once

#include "common.cuh"

namespace irp {

constexpr int kSplineMinSide = 34;  // the row/column passes need W, H >= 34 ...
constexpr int kSplineMaxW = 8192;   // ... and W <= 8192

// Rows wider than 32 lanes x 64 columns take the row pass in segments of at
// most kSegCols source columns: segment s keeps the coefficients of its core
// columns and reads kSegHalo more on each side (except at the frame's edges),
// where its recursions start as if the row ended there.  The error of that
// start is multiplied by |z1|^64 = 3e-37 before it reaches the core, far
// below FP32 rounding.  Cores: [0, kSegCols - kSegHalo), then kSegCore each.
constexpr int kSegCols = 2048;
constexpr int kSegHalo = 64;
constexpr int kSegCore = kSegCols - 2 * kSegHalo;
__host__ __device__ constexpr int row_segments(int W) {
  return W <= kSegCols ? 1 : 1 + (W - (kSegCols - kSegHalo) + kSegCore - 1) / kSegCore;
}
// Core [c0, c1) and source start xs of segment s of a row of W columns.
__host__ __device__ inline void row_segment(int W, int s, int& c0, int& c1, int& xs) {
  if (W <= kSegCols) {
    c0 = 0;
    c1 = W;
    xs = 0;
    return;
  }
  c0 = s == 0 ? 0 : (kSegCols - kSegHalo) + (s - 1) * kSegCore;
  c1 = s == 0 ? kSegCols - kSegHalo : c0 + kSegCore;
  if (c1 > W) c1 = W;
  xs = c0 == 0 ? 0 : c0 - kSegHalo;
}
constexpr int kRowGroup = 16;       // frames per row-pass CTA

// Row pass: rows per CTA for E columns per lane, and its shared memory (the
// block's master rows as float4 plus two raw stages per warp).
constexpr int kRowStages = 2;       // raw-row ring per warp (tasks in flight + 1)
constexpr int kColRows = 64;        // rows per column-pass CTA (32 per warp)
__host__ __device__ constexpr int row_block(int E) { return E == 32 ? 4 : 2; }
// E = 32 also stages each output row per warp, so that it leaves in
// contiguous 512-byte stores.
__host__ __device__ constexpr size_t rows_smem_bytes(int E) {
  return (size_t)row_block(E) * 3 * (E / 4) * 32 * 16 +
         (size_t)8 * kRowStages * (E / 8) * 32 * 16 + (E == 32 ? (size_t)8 * 8 * 32 * 16 : 0);
}

// Row pass over the work items item0 + i * stride, i in [0, count) (row
// block major: item = row0 + rb * frame_groups + g, so stride frame_groups
// walks one frame group's row blocks).
cudaError_t launch_spline_rows(int e, const InlinePlan* inl, const void* plan_dev, int item0,
                               int count, cudaStream_t s, int stride = 1);

// Tile kernel of sets on the row pass: the column recursion, the 16 taps and
// the combine per output tile of kSplineTileCols columns x
// spline_tile_rows(bucket, max_n) rows, over the tiles [item0, item0 + grid).
// Sets of up to IRP_MAX_FRAMES frames combine in registers (bucket = the
// register bucket); deeper sets, to kWideTileMax frames, in groups of G lanes
// per pixel (bucket = wide_tile_bucket(n): 128 for G = 4, 256 for G = 8).
constexpr int kSplineTileCols = 29;  // lane l's horizontal taps reach lane l + 3
constexpr int kWideTileMax = 256;
constexpr size_t kWideTileSmem = 220 * 1024;  // dynamic shared memory of a wide tile CTA
__host__ __device__ constexpr int wide_tile_bucket(int n) { return n <= 128 ? 128 : 256; }
__host__ __device__ constexpr int wide_tile_g(int bucket) { return bucket <= 128 ? 4 : 8; }
// Words per pixel of the wide tile kernel's samples: n, a pad word per 32, odd.
__host__ __device__ constexpr int wide_tile_stride(int n) { return (n + (n + 31) / 32) | 1; }
int spline_tile_rows(int bucket, int max_n);
size_t spline_tile_smem_bytes(int bucket, int max_n);
cudaError_t launch_spline_tile(int bucket, int th, const InlinePlan* inl, const void* plan_dev,
                               int item0, int grid, size_t smem, cudaStream_t s, bool pdl);

// Drops dead intermediate data from L2 without writing it back to HBM
// (discard.global.L2): `count` ranges of `bytes` at p + i * stride, each
// shrunk to the 128-byte lines that lie wholly inside it.
cudaError_t launch_discard_l2(const void* p, size_t bytes, int count, size_t stride,
                              cudaStream_t s);
// Column pass over the work items [item0, item0 + count) (frame major:
// item = colseg0 + (k * row_segments + rs) * col_blocks + cb).
cudaError_t launch_spline_cols(const InlinePlan* inl, const void* plan_dev, int item0, int count,
                               cudaStream_t s);

}  // namespace irp

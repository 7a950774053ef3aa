// spline.h -- launchers of the row and column spline-coefficient passes.
#pragma once

#include "common.cuh"

namespace irp {

constexpr int kSplineMinSide = 34;  // the row/column passes need W, H >= 34 ...
constexpr int kSplineMaxW = 2048;   // ... and W <= 32 lanes x 64 columns
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

cudaError_t launch_spline_rows(int e, const InlinePlan* inl, const void* plan_dev, int nrows,
                               cudaStream_t s);
cudaError_t launch_spline_cols(const InlinePlan* inl, const void* plan_dev, int ncolsegs,
                               cudaStream_t s);

}  // namespace irp

// spline.h -- launchers of the row and column spline-coefficient passes.
#pragma once

#include "common.cuh"

namespace irp {

constexpr int kSplineMinSide = 34;  // the row/column passes need W, H >= 34 ...
constexpr int kSplineMaxW = 2048;   // ... and W <= 32 lanes x 64 columns
constexpr int kRowGroup = 16;       // frames per row-pass CTA (two per warp)

cudaError_t launch_spline_rows(int e, const InlinePlan* inl, const void* plan_dev, int nrows,
                               cudaStream_t s);
cudaError_t launch_spline_cols(const InlinePlan* inl, const void* plan_dev, int ncolsegs,
                               cudaStream_t s);

}  // namespace irp

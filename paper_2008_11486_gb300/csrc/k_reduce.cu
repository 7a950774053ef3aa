// k_reduce.cu -- dispatch of the fused reduction (bucket, geometry, shared
// memory) and the cubic-spline prefilter launch of raw frames.
#include "prefilter.cuh"
#include "reduce_kernels.cuh"
#include "spline.h"

namespace irp {

int reduce_bucket(int n) {
  static const int kBuckets[] = {4, 5, 6, 8, 10, 12, 16, 24, 32, 40, 48, 64};
  for (int b : kBuckets)
    if (n <= b) return b;
  return 64;
}

int tile_cols(int stencil) {
  switch (stencil) {
    case ST_BSPLINE_T: return kSplineTileCols;
    case ST_CUBIC: return StencilShape<ST_CUBIC>::tw;
    case ST_NEAREST: return StencilShape<ST_NEAREST>::tw;
    case ST_BILINEAR: return StencilShape<ST_BILINEAR>::tw;
    case ST_BSPLINE: return StencilShape<ST_BSPLINE>::tw;
    default: return StencilShape<ST_BSPLINE_V>::tw;
  }
}

int rows_per_warp(int bucket, int stencil, int requested) {
  if (requested == rows_per_warp_alt(bucket, stencil)) return requested;
  return rows_per_warp_default(bucket, stencil);
}

int tile_rows(int bucket, int py) { return 8 * py; }

size_t reduce_smem_bytes(int src, int stencil, int py, int max_n, int mwin_f4) {
  return fused_smem_bytes(src, stencil, py, max_n, mwin_f4);
}

cudaError_t launch_reduce(int bucket, int py, int stencil, const InlinePlan* inl,
                          const void* plan_dev, int grid, size_t smem, cudaStream_t s) {
#define IRP_PICK(ST)                                                                   \
  switch (bucket_range(bucket)) {                                                      \
    case 0: return launch_reduce_##ST##_lo(bucket, py, inl, plan_dev, grid, smem, s);  \
    case 1: return launch_reduce_##ST##_mid(bucket, py, inl, plan_dev, grid, smem, s); \
    default: return launch_reduce_##ST##_hi(bucket, py, inl, plan_dev, grid, smem, s); \
  }
  switch (stencil) {
    case ST_NEAREST: IRP_PICK(nearest)
    case ST_BILINEAR: IRP_PICK(bilinear)
    case ST_BSPLINE: IRP_PICK(bspline)
    case ST_CUBIC: IRP_PICK(cubic)
    default: IRP_PICK(bsplinev)
  }
#undef IRP_PICK
}

int reduce_occupancy(int bucket, int py, int stencil, size_t smem) {
#define IRP_PICK(ST)                                                   \
  switch (bucket_range(bucket)) {                                      \
    case 0: return occupancy_reduce_##ST##_lo(bucket, py, smem);       \
    case 1: return occupancy_reduce_##ST##_mid(bucket, py, smem);      \
    default: return occupancy_reduce_##ST##_hi(bucket, py, smem);      \
  }
  switch (stencil) {
    case ST_NEAREST: IRP_PICK(nearest)
    case ST_BILINEAR: IRP_PICK(bilinear)
    case ST_BSPLINE: IRP_PICK(bspline)
    case ST_CUBIC: IRP_PICK(cubic)
    default: IRP_PICK(bsplinev)
  }
#undef IRP_PICK
}

cudaError_t launch_prefilter_raw(const InlinePlan* inl, const void* plan_dev, int grid,
                                 cudaStream_t s) {
  static size_t granted = 0;
  const size_t smem = prefilter_smem_bytes(SRC_RAW);
  cudaError_t e = ensure_smem(k_prefilter<SRC_RAW>, smem, granted);
  if (e != cudaSuccess) return e;
  k_prefilter<SRC_RAW><<<grid, kPrefThreads, smem, s>>>(*inl, plan_dev);
  return cudaGetLastError();
}

}  // namespace irp

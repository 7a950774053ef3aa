// k_reduce_bspline.cu -- fused reduction kernels, bspline stencil, every register bucket.
#include "reduce_kernels.cuh"

namespace irp {

cudaError_t launch_reduce_bspline(int bucket, int py, const InlinePlan* inl, const void* plan_dev,
                                  int grid, size_t smem, cudaStream_t s) {
  return launch_bucket_st<ST_BSPLINE, SRC_F32>(bucket, py, inl, plan_dev, grid, smem, s);
}

int occupancy_reduce_bspline(int bucket, int py, size_t smem) {
  return occupancy_bucket_st<ST_BSPLINE, SRC_F32>(bucket, py, smem);
}

}  // namespace irp

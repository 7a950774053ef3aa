// k_reduce_nearest.cu -- fused reduction kernels, nearest stencil, every register bucket.
#include "reduce_kernels.cuh"

namespace irp {

cudaError_t launch_reduce_nearest(int bucket, int py, const InlinePlan* inl, const void* plan_dev,
                                  int grid, size_t smem, cudaStream_t s) {
  return launch_bucket_st<ST_NEAREST, SRC_RAW>(bucket, py, inl, plan_dev, grid, smem, s);
}

int occupancy_reduce_nearest(int bucket, int py, size_t smem) {
  return occupancy_bucket_st<ST_NEAREST, SRC_RAW>(bucket, py, smem);
}

}  // namespace irp

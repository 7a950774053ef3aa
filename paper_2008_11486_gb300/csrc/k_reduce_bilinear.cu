// k_reduce_bilinear.cu -- fused reduction kernels, bilinear stencil, every register bucket.
#include "reduce_kernels.cuh"

namespace irp {

cudaError_t launch_reduce_bilinear(int bucket, int py, const InlinePlan* inl, const void* plan_dev,
                                  int grid, size_t smem, cudaStream_t s) {
  return launch_bucket_st<ST_BILINEAR, SRC_RAW>(bucket, py, inl, plan_dev, grid, smem, s);
}

int occupancy_reduce_bilinear(int bucket, int py, size_t smem) {
  return occupancy_bucket_st<ST_BILINEAR, SRC_RAW>(bucket, py, smem);
}

}  // namespace irp

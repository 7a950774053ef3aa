// reduce_kernels.cuh -- the fused reduction kernel and its per-bucket launchers
// (each stencil's instantiations live in their own translation unit).
#pragma once

#include "reduce_tile.cuh"

namespace irp {

// One CTA per work item (plain) or persistent CTAs pulling work items from an
// atomic counter in ascending order; the host orders the sets by decreasing
// frame count, so the longest items are handed out first.
// Resident CTAs per SM the register allocation must allow (2 up to 32
// samples per pixel: at most 128 registers per thread).
template <int NMAX>
struct MinBlocks {
  static constexpr int value = NMAX <= 32 ? 2 : 1;
};

template <int NMAX, int STENCIL, int SRC>
__global__ void __launch_bounds__(kThreads, MinBlocks<NMAX>::value)
    k_reduce(const __grid_constant__ InlinePlan inl, const void* plan_dev) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  const PlanView P = make_view(inl, plan_dev);
  const int nitems = P.h->nitems;
  if (!P.h->persistent) {
    if ((int)blockIdx.x < nitems) reduce_tile<NMAX, STENCIL, SRC>(P, blockIdx.x, smem);
    return;
  }
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(P.h->counter, 1u);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= nitems) break;
    reduce_tile<NMAX, STENCIL, SRC>(P, item, smem);
  }
}

// Raises a kernel's dynamic shared-memory opt-in to ``smem`` bytes when it
// needs more than any earlier launch of the same kernel.
template <typename F>
inline cudaError_t ensure_smem(F fn, size_t smem, size_t& granted) {
  // the 48 KB default covers dynamic plus static shared memory: opt in early
  if (smem <= granted || smem <= 47 * 1024) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) granted = smem;
  return e;
}

template <int NMAX, int ST, int SRC>
struct ReduceLauncher {
  static size_t& granted() {
    static size_t g = 0;
    return g;
  }
  static cudaError_t launch(const InlinePlan* inl, const void* plan_dev, int grid, size_t smem,
                            cudaStream_t s) {
    auto fn = k_reduce<NMAX, ST, SRC>;
    cudaError_t e = ensure_smem(fn, smem, granted());
    if (e != cudaSuccess) return e;
    fn<<<grid, kThreads, smem, s>>>(*inl, plan_dev);
    return cudaGetLastError();
  }
  static int occupancy(size_t smem) {
    int blocks = 0;
    if (ensure_smem(k_reduce<NMAX, ST, SRC>, smem, granted()) != cudaSuccess) return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_reduce<NMAX, ST, SRC>, kThreads,
                                                      smem) != cudaSuccess)
      return 1;
    return blocks > 0 ? blocks : 1;
  }
};

#define IRP_FOR_BUCKETS(X) X(4) X(6) X(8) X(10) X(12) X(16) X(24) X(32) X(40) X(48) X(64)

template <int ST, int SRC>
cudaError_t launch_bucket_st(int bucket, const InlinePlan* inl, const void* plan_dev, int grid,
                             size_t smem, cudaStream_t s) {
  switch (bucket) {
#define IRP_CASE(B) \
  case B: return ReduceLauncher<B, ST, SRC>::launch(inl, plan_dev, grid, smem, s);
    IRP_FOR_BUCKETS(IRP_CASE)
#undef IRP_CASE
  }
  return cudaErrorInvalidValue;
}

template <int ST, int SRC>
int occupancy_bucket_st(int bucket, size_t smem) {
  switch (bucket) {
#define IRP_CASE(B) \
  case B: return ReduceLauncher<B, ST, SRC>::occupancy(smem);
    IRP_FOR_BUCKETS(IRP_CASE)
#undef IRP_CASE
  }
  return 1;
}

// per-stencil entry points (k_reduce_<stencil>.cu)
cudaError_t launch_reduce_nearest(int bucket, const InlinePlan* inl, const void* plan_dev, int grid,
                                  size_t smem, cudaStream_t s);
cudaError_t launch_reduce_bilinear(int bucket, const InlinePlan* inl, const void* plan_dev,
                                   int grid, size_t smem, cudaStream_t s);
cudaError_t launch_reduce_bspline(int bucket, const InlinePlan* inl, const void* plan_dev, int grid,
                                  size_t smem, cudaStream_t s);
int occupancy_reduce_nearest(int bucket, size_t smem);
int occupancy_reduce_bilinear(int bucket, size_t smem);
int occupancy_reduce_bspline(int bucket, size_t smem);

}  // namespace irp

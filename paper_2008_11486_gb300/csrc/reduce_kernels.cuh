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

template <int NMAX, int STENCIL, int SRC, int PY>
__global__ void __launch_bounds__(kThreads, MinBlocks<NMAX>::value)
    k_reduce(const __grid_constant__ InlinePlan inl, const void* plan_dev) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  const PlanView P = make_view(inl, plan_dev);
  const int nitems = P.h->nitems;
  if (!P.h->persistent) {
    if ((int)blockIdx.x < nitems) reduce_tile<NMAX, STENCIL, SRC, PY>(P, blockIdx.x, smem);
    return;
  }
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(P.h->counter, 1u);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= nitems) break;
    reduce_tile<NMAX, STENCIL, SRC, PY>(P, item, smem);
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

template <int NMAX, int ST, int SRC, int PY>
struct ReduceLauncher {
  static size_t& granted() {
    static size_t g = 0;
    return g;
  }
  static cudaError_t launch(const InlinePlan* inl, const void* plan_dev, int grid, size_t smem,
                            cudaStream_t s) {
    auto fn = k_reduce<NMAX, ST, SRC, PY>;
    cudaError_t e = ensure_smem(fn, smem, granted());
    if (e != cudaSuccess) return e;
    fn<<<grid, kThreads, smem, s>>>(*inl, plan_dev);
    return cudaGetLastError();
  }
  static int occupancy(size_t smem) {
    int blocks = 0;
    if (ensure_smem(k_reduce<NMAX, ST, SRC, PY>, smem, granted()) != cudaSuccess) return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_reduce<NMAX, ST, SRC, PY>, kThreads,
                                                      smem) != cudaSuccess)
      return 1;
    return blocks > 0 ? blocks : 1;
  }
};

#define IRP_FOR_BUCKETS(X) X(4) X(5) X(6) X(8) X(10) X(12) X(16) X(24) X(32) X(40) X(48) X(64)

// py: rows per warp, rows_per_warp_default(bucket) or rows_per_warp_alt(bucket)
template <int ST, int SRC>
cudaError_t launch_bucket_st(int bucket, int py, const InlinePlan* inl, const void* plan_dev,
                             int grid, size_t smem, cudaStream_t s) {
  const bool alt = py != rows_per_warp_default(bucket);
  switch (bucket) {
#define IRP_CASE(B)                                                                           \
  case B:                                                                                     \
    return alt ? ReduceLauncher<B, ST, SRC, rows_per_warp_alt(B)>::launch(inl, plan_dev, grid, \
                                                                          smem, s)            \
               : ReduceLauncher<B, ST, SRC, rows_per_warp_default(B)>::launch(inl, plan_dev,  \
                                                                              grid, smem, s);
    IRP_FOR_BUCKETS(IRP_CASE)
#undef IRP_CASE
  }
  return cudaErrorInvalidValue;
}

template <int ST, int SRC>
int occupancy_bucket_st(int bucket, int py, size_t smem) {
  const bool alt = py != rows_per_warp_default(bucket);
  switch (bucket) {
#define IRP_CASE(B)                                                               \
  case B:                                                                         \
    return alt ? ReduceLauncher<B, ST, SRC, rows_per_warp_alt(B)>::occupancy(smem) \
               : ReduceLauncher<B, ST, SRC, rows_per_warp_default(B)>::occupancy(smem);
    IRP_FOR_BUCKETS(IRP_CASE)
#undef IRP_CASE
  }
  return 1;
}

// per-stencil entry points (k_reduce_<stencil>.cu)
cudaError_t launch_reduce_nearest(int bucket, int py, const InlinePlan* inl, const void* plan_dev,
                                  int grid, size_t smem, cudaStream_t s);
cudaError_t launch_reduce_bilinear(int bucket, int py, const InlinePlan* inl, const void* plan_dev,
                                   int grid, size_t smem, cudaStream_t s);
cudaError_t launch_reduce_bspline(int bucket, int py, const InlinePlan* inl, const void* plan_dev,
                                  int grid, size_t smem, cudaStream_t s);
int occupancy_reduce_nearest(int bucket, int py, size_t smem);
int occupancy_reduce_bilinear(int bucket, int py, size_t smem);
int occupancy_reduce_bspline(int bucket, int py, size_t smem);

}  // namespace irp

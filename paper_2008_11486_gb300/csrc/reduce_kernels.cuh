// reduce_kernels.cuh -- the fused reduction kernel and its per-bucket launchers
// (each stencil's instantiations live in three translation units by bucket).
#pragma once

#include "reduce_tile.cuh"

namespace irp {

// One CTA per work item (plain) or persistent CTAs pulling work items from an
// atomic counter in ascending order; the host orders the sets by decreasing
// frame count, so the longest items are handed out first.
// Resident CTAs per SM the register allocation must allow (2 up to 40
// samples per pixel, and above with one row per warp: at most 128 registers
// per thread; whether the second CTA fits is then up to the group's shared
// memory).
// The vertical spline taps on filtered rows stage no master window, so up to
// 12 samples per pixel three CTAs fit per SM (at most 85 registers per thread).
template <int NMAX, int STENCIL, int PY>
struct MinBlocks {
  static constexpr int value =
      (STENCIL == ST_BSPLINE_V && NMAX <= 12) ? 3 : (NMAX <= 40 || PY == 1 ? 2 : 1);
};

template <int NMAX, int STENCIL, int SRC, int PY>
__global__ void __launch_bounds__(kThreads, MinBlocks<NMAX, STENCIL, PY>::value)
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

// Register buckets, in three ranges that are compiled in separate
// translation units (k_reduce_<stencil>_<range>.cu) so that the build runs
// in parallel.
#define IRP_BUCKETS_LO(X) X(4) X(5) X(6) X(8) X(10) X(12)
#define IRP_BUCKETS_MID(X) X(16) X(24) X(32)
#define IRP_BUCKETS_HI(X) X(40) X(48) X(64)
#define IRP_FOR_BUCKETS(X) IRP_BUCKETS_LO(X) IRP_BUCKETS_MID(X) IRP_BUCKETS_HI(X)

// The range of a bucket: 0 (4..12), 1 (16..32), 2 (40..64).
inline int bucket_range(int bucket) { return bucket <= 12 ? 0 : (bucket <= 32 ? 1 : 2); }

// Defines launch_reduce_<NAME> and occupancy_reduce_<NAME> over the buckets
// of LIST; py: rows per warp, rows_per_warp_default(bucket, stencil) or
// rows_per_warp_alt(bucket, stencil).
#define IRP_CASE_LAUNCH(B)                                                                    \
  case B:                                                                                     \
    return alt ? ReduceLauncher<B, ST, SRC, rows_per_warp_alt(B, ST)>::launch(inl, plan_dev, grid, \
                                                                          smem, s)            \
               : ReduceLauncher<B, ST, SRC, rows_per_warp_default(B, ST)>::launch(inl, plan_dev,  \
                                                                              grid, smem, s);
#define IRP_CASE_OCC(B)                                                           \
  case B:                                                                         \
    return alt ? ReduceLauncher<B, ST, SRC, rows_per_warp_alt(B, ST)>::occupancy(smem) \
               : ReduceLauncher<B, ST, SRC, rows_per_warp_default(B, ST)>::occupancy(smem);
#define IRP_REDUCE_PART(NAME, STENCIL, SOURCE, LIST)                                          \
  cudaError_t launch_reduce_##NAME(int bucket, int py, const InlinePlan* inl,                 \
                                   const void* plan_dev, int grid, size_t smem,                \
                                   cudaStream_t s) {                                           \
    constexpr int ST = STENCIL, SRC = SOURCE;                                                 \
    const bool alt = py != rows_per_warp_default(bucket, ST);                                     \
    switch (bucket) { LIST(IRP_CASE_LAUNCH) }                                                 \
    return cudaErrorInvalidValue;                                                             \
  }                                                                                           \
  int occupancy_reduce_##NAME(int bucket, int py, size_t smem) {                              \
    constexpr int ST = STENCIL, SRC = SOURCE;                                                 \
    const bool alt = py != rows_per_warp_default(bucket, ST);                                     \
    switch (bucket) { LIST(IRP_CASE_OCC) }                                                    \
    return 1;                                                                                 \
  }

#define IRP_DECLARE_PART(NAME)                                                                \
  cudaError_t launch_reduce_##NAME(int bucket, int py, const InlinePlan* inl,                 \
                                   const void* plan_dev, int grid, size_t smem,                \
                                   cudaStream_t s);                                            \
  int occupancy_reduce_##NAME(int bucket, int py, size_t smem);
IRP_DECLARE_PART(nearest_lo)
IRP_DECLARE_PART(nearest_mid)
IRP_DECLARE_PART(nearest_hi)
IRP_DECLARE_PART(bilinear_lo)
IRP_DECLARE_PART(bilinear_mid)
IRP_DECLARE_PART(bilinear_hi)
IRP_DECLARE_PART(bspline_lo)
IRP_DECLARE_PART(bspline_mid)
IRP_DECLARE_PART(bspline_hi)
IRP_DECLARE_PART(bsplinev_lo)
IRP_DECLARE_PART(bsplinev_mid)
IRP_DECLARE_PART(bsplinev_hi)
IRP_DECLARE_PART(cubic_lo)
IRP_DECLARE_PART(cubic_mid)
IRP_DECLARE_PART(cubic_hi)
#undef IRP_DECLARE_PART

}  // namespace irp

// k_reduce.cu -- fused reduction kernels (plain and persistent) and the
// cubic-spline prefilter launch of raw frames.
#include "prefilter.cuh"
#include "reduce_tile.cuh"

namespace irp {

// One CTA per work item (plain) or persistent CTAs pulling work items from an
// atomic counter in ascending order; the host orders the sets by decreasing
// frame count, so the longest items are handed out first.
template <int NMAX, int STENCIL, int SRC>
__global__ void __launch_bounds__(kThreads)
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

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------
int reduce_bucket(int n) {
  if (n <= 8) return 8;
  if (n <= 16) return 16;
  if (n <= 32) return 32;
  return 64;
}

size_t reduce_smem_bytes(int stencil, int max_n, int mwin_w, int mwin_h) {
  (void)stencil;
  size_t floats = (size_t)max_n * kTilePx + (size_t)kWinRows * kWinStride +
                  3 * (size_t)mwin_w * (size_t)mwin_h;
  return floats * sizeof(float);
}

// Raises the kernel's dynamic shared-memory opt-in to ``smem`` bytes when it
// needs more than any earlier launch of the same instantiation.
template <typename F>
static cudaError_t ensure_smem(F fn, size_t smem, size_t& granted) {
  if (smem <= granted || smem <= 48 * 1024) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) granted = smem;
  return e;
}

template <int NMAX, int ST, int SRC>
static size_t& granted_smem() {
  static size_t g = 0;
  return g;
}

template <int NMAX, int ST, int SRC>
static cudaError_t launch_one(const InlinePlan* inl, const void* plan_dev, int grid,
                              size_t smem, cudaStream_t s) {
  auto fn = k_reduce<NMAX, ST, SRC>;
  cudaError_t e = ensure_smem(fn, smem, granted_smem<NMAX, ST, SRC>());
  if (e != cudaSuccess) return e;
  fn<<<grid, kThreads, smem, s>>>(*inl, plan_dev);
  return cudaGetLastError();
}

template <int ST, int SRC>
static cudaError_t launch_bucket(int bucket, const InlinePlan* inl, const void* plan_dev,
                                 int grid, size_t smem, cudaStream_t s) {
  switch (bucket) {
    case 8: return launch_one<8, ST, SRC>(inl, plan_dev, grid, smem, s);
    case 16: return launch_one<16, ST, SRC>(inl, plan_dev, grid, smem, s);
    case 32: return launch_one<32, ST, SRC>(inl, plan_dev, grid, smem, s);
    default: return launch_one<64, ST, SRC>(inl, plan_dev, grid, smem, s);
  }
}

cudaError_t launch_reduce(int bucket, int stencil, const InlinePlan* inl, const void* plan_dev,
                          int grid, size_t smem, cudaStream_t s) {
  switch (stencil) {
    case ST_NEAREST: return launch_bucket<ST_NEAREST, SRC_RAW>(bucket, inl, plan_dev, grid, smem, s);
    case ST_BILINEAR: return launch_bucket<ST_BILINEAR, SRC_RAW>(bucket, inl, plan_dev, grid, smem, s);
    default: return launch_bucket<ST_BSPLINE, SRC_F32>(bucket, inl, plan_dev, grid, smem, s);
  }
}

template <int NMAX, int ST, int SRC>
static int occ_one(size_t smem) {
  int blocks = 0;
  if (ensure_smem(k_reduce<NMAX, ST, SRC>, smem, granted_smem<NMAX, ST, SRC>()) != cudaSuccess)
    return 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_reduce<NMAX, ST, SRC>, kThreads,
                                                    smem) != cudaSuccess)
    return 1;
  return blocks > 0 ? blocks : 1;
}

template <int ST, int SRC>
static int occ_bucket(int bucket, size_t smem) {
  switch (bucket) {
    case 8: return occ_one<8, ST, SRC>(smem);
    case 16: return occ_one<16, ST, SRC>(smem);
    case 32: return occ_one<32, ST, SRC>(smem);
    default: return occ_one<64, ST, SRC>(smem);
  }
}

int reduce_occupancy(int bucket, int stencil, size_t smem) {
  switch (stencil) {
    case ST_NEAREST: return occ_bucket<ST_NEAREST, SRC_RAW>(bucket, smem);
    case ST_BILINEAR: return occ_bucket<ST_BILINEAR, SRC_RAW>(bucket, smem);
    default: return occ_bucket<ST_BSPLINE, SRC_F32>(bucket, smem);
  }
}

cudaError_t launch_prefilter_raw(const InlinePlan* inl, const void* plan_dev, int grid,
                                 cudaStream_t s) {
  static size_t granted = 0;
  const size_t smem = prefilter_smem_bytes();
  cudaError_t e = ensure_smem(k_prefilter<SRC_RAW>, smem, granted);
  if (e != cudaSuccess) return e;
  k_prefilter<SRC_RAW><<<grid, kThreads, smem, s>>>(*inl, plan_dev);
  return cudaGetLastError();
}

}  // namespace irp

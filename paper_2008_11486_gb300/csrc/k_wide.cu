// k_wide.cu -- combination of an aligned stack of more frames than the
// register buckets hold (Sec. 2.1 co-adding; the paper's sets reach 180
// frames per band): one CTA per 32 pixels of an output row, one warp per
// pixel.
#include "unfused.h"
#include "wide.cuh"

namespace irp {

// The CTA copies its [n][32] slab of the stack into shared memory (each
// frame's 32 pixels are one 128-byte row segment), then its 8 warps take the
// 32 pixels in turn: load, sort (the sorted run replaces the samples in
// shared memory, where the order statistics are read), clip, and write the
// results as one row.
template <int J, bool F16>
__global__ void __launch_bounds__(kWideThreads) k_combine_wide(CombineArgs a, int tiles_x) {
  extern __shared__ float s_wide[];
  __shared__ float s_mean[32], s_median[32];
  __shared__ int s_kept[32];
  using SM = WideSmem<J>;
  const int tx = blockIdx.x % tiles_x;
  const int y = blockIdx.x / tiles_x;
  const int x0 = tx * 32;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const float kInf = __int_as_float(0x7f800000);
  const int n = a.n;
  // sample of frame k at stack offset o: +inf when invalid (NaN or masked)
  auto load = [&](int k, int64_t o) -> float {
    float v;
    if (F16)
      v = __fmaf_rn(__half2float(((const __half*)a.stack)[o]), __ldg(a.scale + k),
                    __ldg(a.offset + k));
    else
      v = __ldg((const float*)a.stack + o);
    if (a.valid && !__ldg(a.valid + o)) v = kInf;
    return (v == v) ? v : kInf;
  };
  {
    // staging: thread (warp, lane) copies frames warp, warp + 8, ... of pixel lane
    const int x = x0 + lane;
    const bool xin = x < a.W;
    const int64_t o0 = (int64_t)y * a.pitch + x;
    constexpr int kBatch = 16;  // loads in flight per thread
    for (int k0 = warp; k0 < n; k0 += 8 * kBatch) {
      float v[kBatch];
#pragma unroll
      for (int b = 0; b < kBatch; ++b) {
        const int k = k0 + 8 * b;
        v[b] = (xin && k < n) ? load(k, (int64_t)k * a.fstride + o0) : kInf;
      }
#pragma unroll
      for (int b = 0; b < kBatch; ++b) {
        const int k = k0 + 8 * b;
        if (k < n) s_wide[SM::at(lane, k)] = v[b];
      }
    }
  }
  __syncthreads();
#pragma unroll 1
  for (int p = warp; p < 32; p += 8) {
    if (x0 + p >= a.W) break;
    float* const col = s_wide + SM::at(p, 0);  // this pixel's samples
    float v[J];
    int cnt = 0;
#pragma unroll
    for (int i = 0; i < J; ++i) {
      const int e = lane * J + i;
      v[i] = e < n ? col[lane * (J + 1) + i] : kInf;
      cnt += v[i] < kInf ? 1 : 0;
    }
    const int m = __reduce_add_sync(0xffffffffu, cnt);
    if (m > 0) warp_bitonic_sort<J>(v, lane);
    // the sorted run replaces the pixel's samples (sample e at col[e + e / J])
    __syncwarp();
#pragma unroll
    for (int i = 0; i < J; ++i) col[lane * (J + 1) + i] = v[i];
    __syncwarp();
    const WideOut o = wide_combine<J>(v, col, m, a.clip, lane);
    if (lane == 0) {
      s_mean[p] = o.mean;
      s_median[p] = o.median;
      s_kept[p] = o.kept;
    }
    if (a.reject_out) {  // debug output: the frames' samples again, in frame order
      const int x = x0 + p;
      const int64_t o0 = (int64_t)y * a.pitch + x;
      for (int k = lane; k < n; k += 32) {
        const float val = load(k, (int64_t)k * a.fstride + o0);
        const bool rej = (val < kInf) & ((val < o.lo_val) | (val > o.hi_val));
        a.reject_out[((int64_t)k * a.H + y) * a.out_pitch + x] = rej ? 1 : 0;
      }
    }
  }
  __syncthreads();
  if (t < 32 && x0 + t < a.W) {
    const int64_t oi = (int64_t)y * a.out_pitch + x0 + t;
    if (a.mean_out) a.mean_out[oi] = s_mean[t];
    if (a.median_out) a.median_out[oi] = s_median[t];
    if (a.nkept_out) a.nkept_out[oi] = (uint16_t)s_kept[t];
  }
}

template <int J, bool F16>
static cudaError_t combine_wide_j(const CombineArgs& a, cudaStream_t s) {
  static size_t granted = 0;
  const size_t smem = WideSmem<J>::kBytes;
  auto fn = k_combine_wide<J, F16>;
  if (smem > granted && smem > 47 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    granted = smem;
  }
  const int tiles_x = (a.W + 31) / 32;
  const int64_t grid = (int64_t)tiles_x * a.H;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  fn<<<(unsigned)grid, kWideThreads, smem, s>>>(a, tiles_x);
  return cudaGetLastError();
}

template <bool F16>
static cudaError_t combine_wide_f(const CombineArgs& a, cudaStream_t s) {
  switch (wide_j(a.n)) {
    case 4: return combine_wide_j<4, F16>(a, s);
    case 8: return combine_wide_j<8, F16>(a, s);
    case 16: return combine_wide_j<16, F16>(a, s);
    default: return combine_wide_j<32, F16>(a, s);
  }
}

cudaError_t launch_combine_wide(const CombineArgs& a, bool f16, cudaStream_t s) {
  if (a.n < 1 || a.n > kWideMaxFrames) return cudaErrorInvalidValue;
  return f16 ? combine_wide_f<true>(a, s) : combine_wide_f<false>(a, s);
}

}  // namespace irp

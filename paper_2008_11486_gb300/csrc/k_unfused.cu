// k_unfused.cu -- the three steps as separate kernels, with the aligned stack
// materialised in HBM as FP32 or as FP16 with a per-frame scale and offset,
// and the FP64 frame-wide sums that choose that scaling.
#include <float.h>

#include "combine.cuh"
#include "prefilter.cuh"
#include "reduce_kernels.cuh"
#include "unfused.h"

namespace irp {

// ---------------------------------------------------------------------------
// FP64 frame-wide sums (sky level, flat normalisation).  Each block reduces a
// grid-stride share of one frame with warp shuffles and adds one FP64 partial
// per block; min/max use order-preserving integer keys.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int float_key(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float key_float(int k) {
  return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

struct StatsAcc {
  double s, q;
  long long c;
  float mn, mx;
};

__device__ __forceinline__ void stats_commit(StatsAcc a, double* sum, double* sumsq,
                                             long long* count, int* min_key, int* max_key) {
  __shared__ double sh_s[kThreads / 32], sh_q[kThreads / 32];
  __shared__ long long sh_c[kThreads / 32];
  __shared__ float sh_mn[kThreads / 32], sh_mx[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  a.s = warp_sum(a.s);
  a.q = warp_sum(a.q);
  a.c = warp_sum(a.c);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a.mn = fminf(a.mn, __shfl_down_sync(0xffffffffu, a.mn, o));
    a.mx = fmaxf(a.mx, __shfl_down_sync(0xffffffffu, a.mx, o));
  }
  if (lane == 0) {
    sh_s[warp] = a.s;
    sh_q[warp] = a.q;
    sh_c[warp] = a.c;
    sh_mn[warp] = a.mn;
    sh_mx[warp] = a.mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0, q = 0.0;
    long long c = 0;
    float mn = FLT_MAX, mx = -FLT_MAX;
    for (int w = 0; w < kThreads / 32; ++w) {
      s += sh_s[w];
      q += sh_q[w];
      c += sh_c[w];
      mn = fminf(mn, sh_mn[w]);
      mx = fmaxf(mx, sh_mx[w]);
    }
    atomicAdd(sum, s);
    if (sumsq) atomicAdd(sumsq, q);
    if (count) atomicAdd((unsigned long long*)count, (unsigned long long)c);
    if (min_key) atomicMin(min_key, float_key(mn));
    if (max_key) atomicMax(max_key, float_key(mx));
  }
}

__global__ void k_stats_init(FrameStats* st, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    st[i].sum = 0.0;
    st[i].sumsq = 0.0;
    st[i].count = 0;
    st[i].min_key = 0x7fffffff;
    st[i].max_key = (int)0x80000000;
  }
}

// Sums of calibrated raw frames (FP16 scaling needs them before quantising).
__global__ void __launch_bounds__(kThreads)
    k_stats_raw(CalibArgs a, FrameStats* st) {
  const int k = blockIdx.y + a.k0;
  const uint16_t* raw = a.raw + (int64_t)k * a.raw_frame_stride;
  const float t = a.t[blockIdx.y];
  const float flat_norm = a.flat_sum ? (float)(*a.flat_sum / ((double)a.W * a.H)) : 1.0f;
  StatsAcc acc{0.0, 0.0, 0, FLT_MAX, -FLT_MAX};
  const int64_t P = (int64_t)a.W * a.H;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < P;
       i += (int64_t)gridDim.x * kThreads) {
    const int y = (int)(i / a.W), x = (int)(i - (int64_t)y * a.W);
    const int64_t m = (int64_t)y * a.master_pitch + x;
    const float rf = inv_flat(__ldg(a.flat + m), flat_norm, a.status);
    const float v = calibrate_px(__ldg(raw + (int64_t)y * a.raw_pitch + x), __ldg(a.bias + m),
                                 __ldg(a.dark + m), t, rf);
    acc.s += (double)v;
    acc.q += (double)v * (double)v;
    acc.c += 1;
    acc.mn = fminf(acc.mn, v);
    acc.mx = fmaxf(acc.mx, v);
  }
  stats_commit(acc, &st[k].sum, &st[k].sumsq, &st[k].count, &st[k].min_key, &st[k].max_key);
}

// Sums of F32 / F16-scaled frames, NaN skipped (also the flat master).
template <bool F16>
__global__ void __launch_bounds__(kThreads)
    k_stats_frames(const void* frames, int64_t pitch, int64_t fstride, int W, int H,
                   const float* scale, const float* offset, double* sum, double* sumsq,
                   long long* count, FrameStats* st) {
  const int k = blockIdx.y;
  StatsAcc acc{0.0, 0.0, 0, FLT_MAX, -FLT_MAX};
  const int64_t P = (int64_t)W * H;
  const float sc = (F16 && scale) ? scale[k] : 1.0f, of = (F16 && offset) ? offset[k] : 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < P;
       i += (int64_t)gridDim.x * kThreads) {
    const int y = (int)(i / W), x = (int)(i - (int64_t)y * W);
    const int64_t o = (int64_t)k * fstride + (int64_t)y * pitch + x;
    float v;
    if (F16) {
      v = __fmaf_rn(__half2float(((const __half*)frames)[o]), sc, of);
    } else {
      v = __ldg((const float*)frames + o);
    }
    if (v == v) {
      acc.s += (double)v;
      acc.q += (double)v * (double)v;
      acc.c += 1;
      acc.mn = fminf(acc.mn, v);
      acc.mx = fmaxf(acc.mx, v);
    }
  }
  if (st)
    stats_commit(acc, &st[k].sum, &st[k].sumsq, &st[k].count, &st[k].min_key, &st[k].max_key);
  else
    stats_commit(acc, sum + k, sumsq ? sumsq + k : nullptr, count ? count + k : nullptr, nullptr,
                 nullptr);
}

// offset = FP64 mean of the frame; scale = the power of two with
// max |v - offset| / scale <= kF16Range (headroom for spline overshoot).
__global__ void k_f16_scaling(const FrameStats* st, int n, float* scale, float* offset) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double mean = st[k].count > 0 ? st[k].sum / (double)st[k].count : 0.0;
  const float off = (float)mean;
  const float mn = key_float(st[k].min_key), mx = key_float(st[k].max_key);
  const float amax = fmaxf(fabsf(mx - off), fabsf(off - mn));
  int e = 0;
  if (amax > 0.0f && isfinite(amax)) e = (int)ceilf(log2f(amax / kF16Range));
  e = max(min(e, 100), -24);
  offset[k] = off;
  scale[k] = ldexpf(1.0f, e);
}

// ---------------------------------------------------------------------------
// Calibration (Sec. 2.1), one thread per pixel.
// ---------------------------------------------------------------------------
template <bool F16>
__global__ void __launch_bounds__(kThreads) k_calibrate(CalibArgs a, void* out, int64_t out_pitch,
                                                        int64_t out_fstride, const float* scale,
                                                        const float* offset) {
  const int x = blockIdx.x * kThreads + threadIdx.x;
  const int y = blockIdx.y;
  const int k = blockIdx.z + a.k0;
  if (x >= a.W) return;
  const float flat_norm = a.flat_sum ? (float)(*a.flat_sum / ((double)a.W * a.H)) : 1.0f;
  const int64_t m = (int64_t)y * a.master_pitch + x;
  const float rf = inv_flat(__ldg(a.flat + m), flat_norm, a.status);
  const uint16_t q = __ldg(a.raw + (int64_t)k * a.raw_frame_stride + (int64_t)y * a.raw_pitch + x);
  const float v = calibrate_px(q, __ldg(a.bias + m), __ldg(a.dark + m), a.t[blockIdx.z], rf);
  const int64_t o = (int64_t)k * out_fstride + (int64_t)y * out_pitch + x;
  if (F16) {
    const float inv = 1.0f / scale[k];  // exact: the scale is a power of two
    ((__half*)out)[o] = __float2half_rn(__fmul_rn(__fsub_rn(v, offset[k]), inv));
  } else {
    ((float*)out)[o] = v;
  }
}

// ---------------------------------------------------------------------------
// Shift (Sec. 2.1 alignment) of calibrated frames, one thread per output
// pixel; taps are read from the frame (nearest, bilinear) or from the frame's
// spline coefficients (cubic spline, mirror-extended).
// ---------------------------------------------------------------------------
template <int ST, bool F16>
__global__ void __launch_bounds__(kThreads) k_shift(ShiftArgs a) {
  const int x = blockIdx.x * kThreads + threadIdx.x;
  const int y = blockIdx.y;
  const int kl = blockIdx.z;
  if (x >= a.W) return;
  const FrameDesc& F = a.frames[kl];
  const int k = a.k0 + kl;
  const bool ok = (x >= F.vx0) & (x <= F.vx1) & (y >= F.vy0) & (y <= F.vy1);
  float val = __int_as_float(0x7fc00000);
  if (ok) {
    const int i0 = x + F.ox, j0 = y + F.oy;
    if (ST == ST_BSPLINE) {
      // padded coefficient frame: (x, y) at (y + 2) * pitch + x + 2
      const float* c = F.coef;
      float acc = 0.0f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = min(max(j0 + q, -2), a.H + 1);
        const float* row = c + (int64_t)(j + 2) * a.coef_pitch + 2;
        float h = 0.0f;
#pragma unroll
        for (int p = 0; p < 4; ++p) h = __fmaf_rn(F.wx[p], __ldg(row + min(max(i0 + p, -2), a.W + 1)), h);
        acc = __fmaf_rn(F.wy[q], h, acc);
      }
      val = acc;
    } else {
      auto at = [&](int i, int j) -> float {
        const int64_t o = (int64_t)k * a.in_fstride + (int64_t)j * a.in_pitch + i;
        if (F16) return __half2float(((const __half*)a.in)[o]);
        return __ldg((const float*)a.in + o);
      };
      if (ST == ST_NEAREST) {
        val = at(i0, j0);
      } else {
        // zero-weight taps are not read (they may lie outside the frame)
        const float p00 = at(i0, j0);
        const float p10 = F.fx != 0.0f ? at(i0 + 1, j0) : p00;
        const float h0 = __fmaf_rn(F.fx, __fsub_rn(p10, p00), p00);
        float h1 = h0;
        if (F.fy != 0.0f) {
          const float p01 = at(i0, j0 + 1);
          const float p11 = F.fx != 0.0f ? at(i0 + 1, j0 + 1) : p01;
          h1 = __fmaf_rn(F.fx, __fsub_rn(p11, p01), p01);
        }
        val = __fmaf_rn(F.fy, __fsub_rn(h1, h0), h0);
      }
    }
  }
  const int64_t o = (int64_t)k * a.out_fstride + (int64_t)y * a.out_pitch + x;
  if (F16)
    ((__half*)a.out)[o] = __float2half_rn(val);
  else
    ((float*)a.out)[o] = val;
  if (a.valid_out) a.valid_out[o] = ok ? 1 : 0;
}

// ---------------------------------------------------------------------------
// Combine (Sec. 2.1 co-adding) of a materialised stack, one thread per pixel.
// ---------------------------------------------------------------------------
template <int NMAX, bool F16>
__global__ void __launch_bounds__(kThreads) k_combine(CombineArgs a) {
  const int x = blockIdx.x * kThreads + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= a.W) return;
  const float kInf = __int_as_float(0x7f800000);
  auto load = [&](int k) -> float {
    const int64_t o = (int64_t)k * a.fstride + (int64_t)y * a.pitch + x;
    float v;
    if (F16)
      v = __fmaf_rn(__half2float(((const __half*)a.stack)[o]), __ldg(a.scale + k), __ldg(a.offset + k));
    else
      v = __ldg((const float*)a.stack + o);
    if (a.valid && !a.valid[o]) v = kInf;
    return (v == v) ? v : kInf;
  };
  float s[NMAX];
  int m = 0;
#pragma unroll
  for (int j = 0; j < NMAX; ++j) {
    s[j] = (j < a.n) ? load(j) : kInf;
    m += (s[j] < kInf) ? 1 : 0;
  }
  sort_network<NMAX>(s);
  const CombineOut o = combine_sorted<NMAX>(s, m, a.clip);
  const int64_t oi = (int64_t)y * a.out_pitch + x;
  if (a.mean_out) a.mean_out[oi] = o.mean;
  if (a.median_out) a.median_out[oi] = o.median;
  if (a.nkept_out) a.nkept_out[oi] = (uint16_t)o.kept;
  if (a.reject_out) {
    for (int k = 0; k < a.n; ++k) {
      const float v = load(k);
      const bool rej = (v < kInf) & ((v < o.lo_val) | (v > o.hi_val));
      a.reject_out[((int64_t)k * a.H + y) * a.out_pitch + x] = rej ? 1 : 0;
    }
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static int stats_blocks(int64_t P) {
  int64_t b = (P + kThreads * 8 - 1) / (kThreads * 8);
  return (int)(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

cudaError_t launch_stats_init(FrameStats* st, int n, cudaStream_t s) {
  k_stats_init<<<(n + 255) / 256, 256, 0, s>>>(st, n);
  return cudaGetLastError();
}

cudaError_t launch_stats_raw(const CalibArgs& a, int nk, FrameStats* st, cudaStream_t s) {
  dim3 grid(stats_blocks((int64_t)a.W * a.H), nk);
  k_stats_raw<<<grid, kThreads, 0, s>>>(a, st);
  return cudaGetLastError();
}

cudaError_t launch_stats_frames(const void* frames, int64_t pitch, int64_t fstride, int W, int H,
                                int n, bool f16, const float* scale, const float* offset,
                                double* sum, double* sumsq, long long* count, FrameStats* st,
                                cudaStream_t s) {
  dim3 grid(stats_blocks((int64_t)W * H), n);
  if (f16)
    k_stats_frames<true><<<grid, kThreads, 0, s>>>(frames, pitch, fstride, W, H, scale, offset,
                                                   sum, sumsq, count, st);
  else
    k_stats_frames<false><<<grid, kThreads, 0, s>>>(frames, pitch, fstride, W, H, scale, offset,
                                                    sum, sumsq, count, st);
  return cudaGetLastError();
}

cudaError_t launch_f16_scaling(const FrameStats* st, int n, float* scale, float* offset,
                               cudaStream_t s) {
  k_f16_scaling<<<(n + 127) / 128, 128, 0, s>>>(st, n, scale, offset);
  return cudaGetLastError();
}

cudaError_t launch_calibrate(const CalibArgs& a, int nk, bool f16, void* out, int64_t out_pitch,
                             int64_t out_fstride, const float* scale, const float* offset,
                             cudaStream_t s) {
  dim3 grid((a.W + kThreads - 1) / kThreads, a.H, nk);
  if (f16)
    k_calibrate<true><<<grid, kThreads, 0, s>>>(a, out, out_pitch, out_fstride, scale, offset);
  else
    k_calibrate<false><<<grid, kThreads, 0, s>>>(a, out, out_pitch, out_fstride, scale, offset);
  return cudaGetLastError();
}

template <int ST>
static cudaError_t shift_st(const ShiftArgs& a, int nk, bool f16, cudaStream_t s) {
  dim3 grid((a.W + kThreads - 1) / kThreads, a.H, nk);
  if (f16)
    k_shift<ST, true><<<grid, kThreads, 0, s>>>(a);
  else
    k_shift<ST, false><<<grid, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_shift(const ShiftArgs& a, int nk, int stencil, bool f16, cudaStream_t s) {
  switch (stencil) {
    case ST_NEAREST: return shift_st<ST_NEAREST>(a, nk, f16, s);
    case ST_BILINEAR: return shift_st<ST_BILINEAR>(a, nk, f16, s);
    default: return shift_st<ST_BSPLINE>(a, nk, f16, s);
  }
}

cudaError_t launch_prefilter_frames(const InlinePlan* inl, int grid, bool f16, cudaStream_t s) {
  static size_t granted32 = 0, granted16 = 0;
  const size_t smem = prefilter_smem_bytes(SRC_F32);
  cudaError_t e;
  if (f16) {
    e = ensure_smem(k_prefilter<SRC_F16>, smem, granted16);
    if (e == cudaSuccess) k_prefilter<SRC_F16><<<grid, kPrefThreads, smem, s>>>(*inl, nullptr);
  } else {
    e = ensure_smem(k_prefilter<SRC_F32>, smem, granted32);
    if (e == cudaSuccess) k_prefilter<SRC_F32><<<grid, kPrefThreads, smem, s>>>(*inl, nullptr);
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int NMAX>
static cudaError_t combine_n(const CombineArgs& a, bool f16, cudaStream_t s) {
  dim3 grid((a.W + kThreads - 1) / kThreads, a.H);
  if (f16)
    k_combine<NMAX, true><<<grid, kThreads, 0, s>>>(a);
  else
    k_combine<NMAX, false><<<grid, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_combine(const CombineArgs& a, bool f16, cudaStream_t s) {
  switch (reduce_bucket(a.n)) {
#define IRP_CASE(B) \
  case B: return combine_n<B>(a, f16, s);
    IRP_FOR_BUCKETS(IRP_CASE)
#undef IRP_CASE
  }
  return cudaErrorInvalidValue;
}

}  // namespace irp

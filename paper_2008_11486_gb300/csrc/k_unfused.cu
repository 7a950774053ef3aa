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

// A thread's partial sums over one row in FP32 with exact error terms: each
// addition is split by TwoSum into its rounded sum and its rounding error,
// and each square by one fused multiply-add into rn(v v) and its remainder;
// the (small) error terms are summed in FP32.  A row's partials (at most
// W / 256 values) are then added into FP64, so the frame sum carries FP64
// accuracy at the FP32 arithmetic rate.
struct RowPartial {
  float s, es, q, eq;
};

__device__ __forceinline__ void two_sum_add(float& s, float& e, float v) {
  const float t = __fadd_rn(s, v);
  const float bp = __fsub_rn(t, s);
  e = __fadd_rn(e, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp)));
  s = t;
}

__device__ __forceinline__ void row_add(RowPartial& r, float v) {
  two_sum_add(r.s, r.es, v);
  const float p = __fmul_rn(v, v);
  two_sum_add(r.q, r.eq, p);
  r.eq = __fadd_rn(r.eq, __fmaf_rn(v, v, -p));
}

__device__ __forceinline__ void row_flush(StatsAcc& acc, const RowPartial& r) {
  acc.s += (double)r.s + (double)r.es;
  acc.q += (double)r.q + (double)r.eq;
}


// Sums of calibrated raw frames (FP16 scaling needs them before quantising).
// Block b covers frame b % nk and the row block b / nk: consecutive blocks
// share the row block's masters, which are then read from L2 for all frames
// but the first.
__global__ void __launch_bounds__(kThreads)
    k_stats_raw(CalibArgs a, int nk, FrameStats* st) {
  const int kl = blockIdx.x % nk, rb = blockIdx.x / nk;
  const int k = kl + a.k0;
  const uint16_t* raw = a.raw + (int64_t)k * a.raw_frame_stride;
  const float t = a.t[kl];
  const float flat_norm = a.flat_sum ? (float)(*a.flat_sum / ((double)a.W * a.H)) : 1.0f;
  StatsAcc acc{0.0, 0.0, 0, FLT_MAX, -FLT_MAX};
  const int R = stats_rows(a.W, a.H);
  const int y1 = min(a.H, (rb + 1) * R);
  for (int y = rb * R; y < y1; ++y) {
    RowPartial r{0.0f, 0.0f, 0.0f, 0.0f};
    const uint16_t* rr = raw + (int64_t)y * a.raw_pitch;
    const int64_t mrow = (int64_t)y * a.master_pitch;
    if (a.vec) {
      for (int x = 4 * threadIdx.x; x < a.W; x += 4 * kThreads) {
        const uint2 q = __ldg((const uint2*)(rr + x));
        const float4 b = __ldg((const float4*)(a.bias + mrow + x));
        const float4 d = __ldg((const float4*)(a.dark + mrow + x));
        const float4 f = __ldg((const float4*)(a.flat + mrow + x));
        const float v[4] = {
            calibrate_pxf(u16_lo_to_float(q.x), b.x, d.x, t, inv_flat(f.x, flat_norm, a.status)),
            calibrate_pxf(u16_hi_to_float(q.x), b.y, d.y, t, inv_flat(f.y, flat_norm, a.status)),
            calibrate_pxf(u16_lo_to_float(q.y), b.z, d.z, t, inv_flat(f.z, flat_norm, a.status)),
            calibrate_pxf(u16_hi_to_float(q.y), b.w, d.w, t, inv_flat(f.w, flat_norm, a.status))};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          row_add(r, v[e]);
          acc.mn = fminf(acc.mn, v[e]);
          acc.mx = fmaxf(acc.mx, v[e]);
        }
        acc.c += 4;
      }
      row_flush(acc, r);
      continue;
    }
    for (int x = threadIdx.x; x < a.W; x += kThreads) {
      const float rf = inv_flat(__ldg(a.flat + mrow + x), flat_norm, a.status);
      const float v = calibrate_px(__ldg(rr + x), __ldg(a.bias + mrow + x),
                                   __ldg(a.dark + mrow + x), t, rf);
      row_add(r, v);
      acc.c += 1;
      acc.mn = fminf(acc.mn, v);
      acc.mx = fmaxf(acc.mx, v);
    }
    row_flush(acc, r);
  }
  stats_commit(acc, &st[k].sum, &st[k].sumsq, &st[k].count, &st[k].min_key, &st[k].max_key);
}

// Per-frame normalisation: the FP64 sum of every calibrated raw frame of a
// plan's sets.  Block b covers frame b % nframes and its row block
// b / nframes (rows of stats_rows(W, H) each); blocks past a set's rows exit.
__global__ void __launch_bounds__(kThreads)
    k_frame_means(const __grid_constant__ InlinePlan inl, const void* plan_dev) {
  const PlanView P = make_view(inl, plan_dev);
  const int nf = P.h->nframes;
  const int f = blockIdx.x % nf, rb = blockIdx.x / nf;
  int si = 0;
  {
    int lo = 0, hi = P.h->nsets - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (P.sets[mid].frame0 <= f) lo = mid; else hi = mid - 1;
    }
    si = lo;
  }
  const SetDesc& S = P.sets[si];
  const FrameDesc& F = P.frames[f];
  const int W = S.W, H = S.H;
  const int R = stats_rows(W, H);
  if (rb * R >= H || !F.norm) return;
  const float flat_norm = S.flat_sum ? (float)(*S.flat_sum / ((double)W * H)) : 1.0f;
  const uint16_t* raw = (const uint16_t*)F.src;
  StatsAcc acc{0.0, 0.0, 0, FLT_MAX, -FLT_MAX};
  const int y1 = min(H, (rb + 1) * R);
  for (int y = rb * R; y < y1; ++y) {
    RowPartial r{0.0f, 0.0f, 0.0f, 0.0f};
    const uint16_t* rr = raw + (int64_t)y * S.src_pitch;
    const int64_t mrow = (int64_t)y * S.master_pitch;
    for (int x = threadIdx.x; x < W; x += kThreads) {
      const float rf = inv_flat(__ldg(S.flat + mrow + x), flat_norm, P.h->status);
      row_add(r, calibrate_px(__ldg(rr + x), __ldg(S.bias + mrow + x), __ldg(S.dark + mrow + x),
                              F.t, rf));
    }
    row_flush(acc, r);
  }
  stats_commit(acc, &F.norm->sum, nullptr, nullptr, nullptr, nullptr);
}

// The factors of every frame from the sums: frame 0 of the set (norm_ref) is
// the reference.
__global__ void k_frame_norm_factors(const __grid_constant__ InlinePlan inl, const void* plan_dev) {
  const PlanView P = make_view(inl, plan_dev);
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= P.h->nframes) return;
  int si = 0;
  {
    int lo = 0, hi = P.h->nsets - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (P.sets[mid].frame0 <= f) lo = mid; else hi = mid - 1;
    }
    si = lo;
  }
  const SetDesc& S = P.sets[si];
  FrameNorm* rec = P.frames[f].norm;
  if (!rec || !S.norm_ref) return;
  const double px = (double)S.W * S.H;
  const double mk = rec->sum / px, m0 = S.norm_ref->sum / px;
  float na = 1.0f, nz = 0.0f;
  if (P.h->frame_norm == 1) {
    nz = (float)(m0 - mk);
  } else {
    if (!(mk != 0.0) || !isfinite(mk) || !isfinite(m0)) {
      latch_status(P.h->status, IRP_ERR_BAD_STATISTIC);
      na = __int_as_float(0x7fffffff);
    } else {
      na = (float)(m0 / mk);
    }
  }
  rec->na = na;
  rec->nz = nz;
}

// Sums of F32 / F16-scaled frames, NaN skipped (also the flat master).
template <bool F16>
__global__ void __launch_bounds__(kThreads)
    k_stats_frames(const void* frames, int64_t pitch, int64_t fstride, int W, int H, int n,
                   const float* scale, const float* offset, double* sum, double* sumsq,
                   long long* count, FrameStats* st) {
  const int k = blockIdx.x % n, rb = blockIdx.x / n;
  StatsAcc acc{0.0, 0.0, 0, FLT_MAX, -FLT_MAX};
  const float sc = (F16 && scale) ? scale[k] : 1.0f, of = (F16 && offset) ? offset[k] : 0.0f;
  const int R = stats_rows(W, H);
  const int y1 = min(H, (rb + 1) * R);
  for (int y = rb * R; y < y1; ++y) {
    RowPartial r{0.0f, 0.0f, 0.0f, 0.0f};
    const int64_t o = (int64_t)k * fstride + (int64_t)y * pitch;
    for (int x = threadIdx.x; x < W; x += kThreads) {
      float v;
      if (F16) {
        v = __fmaf_rn(__half2float(((const __half*)frames)[o + x]), sc, of);
      } else {
        v = __ldg((const float*)frames + o + x);
      }
      if (v == v) {
        row_add(r, v);
        acc.c += 1;
        acc.mn = fminf(acc.mn, v);
        acc.mx = fmaxf(acc.mx, v);
      }
    }
    row_flush(acc, r);
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
// Calibration (Sec. 2.1).  Block b covers frame b % nk of one row segment of
// 1024 pixels (four per thread, coalesced); consecutive blocks share the
// segment's masters, read from L2 for all frames but the first.
// ---------------------------------------------------------------------------
constexpr int kCalibSeg = 4 * kThreads;

template <bool F16>
__global__ void __launch_bounds__(kThreads) k_calibrate(CalibArgs a, int nk, void* out,
                                                        int64_t out_pitch, int64_t out_fstride,
                                                        const float* scale,
                                                        const float* offset) {
  const int kl = blockIdx.x % nk;
  const int64_t seg = blockIdx.x / nk;
  const int nseg = (a.W + kCalibSeg - 1) / kCalibSeg;
  const int y = (int)(seg / nseg);
  const int xs = (int)(seg - (int64_t)y * nseg) * kCalibSeg;
  const int k = kl + a.k0;
  const float flat_norm = a.flat_sum ? (float)(*a.flat_sum / ((double)a.W * a.H)) : 1.0f;
  const float t = a.t[kl];
  const uint16_t* rr = a.raw + (int64_t)k * a.raw_frame_stride + (int64_t)y * a.raw_pitch;
  const int64_t mrow = (int64_t)y * a.master_pitch;
  const int64_t orow = (int64_t)k * out_fstride + (int64_t)y * out_pitch;
  float inv = 1.0f, off = 0.0f;
  if (F16) {
    inv = 1.0f / scale[k];  // exact: the scale is a power of two
    off = offset[k];
  }
  if (a.vec) {
    const int x = xs + 4 * threadIdx.x;
    if (x >= a.W) return;
    const uint2 q = __ldg((const uint2*)(rr + x));
    const float4 b = __ldg((const float4*)(a.bias + mrow + x));
    const float4 d = __ldg((const float4*)(a.dark + mrow + x));
    const float4 f = __ldg((const float4*)(a.flat + mrow + x));
    float v[4] = {
        calibrate_pxf(u16_lo_to_float(q.x), b.x, d.x, t, inv_flat(f.x, flat_norm, a.status)),
        calibrate_pxf(u16_hi_to_float(q.x), b.y, d.y, t, inv_flat(f.y, flat_norm, a.status)),
        calibrate_pxf(u16_lo_to_float(q.y), b.z, d.z, t, inv_flat(f.z, flat_norm, a.status)),
        calibrate_pxf(u16_hi_to_float(q.y), b.w, d.w, t, inv_flat(f.w, flat_norm, a.status))};
    if (F16) {
      __half h[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) h[e] = __float2half_rn(__fmul_rn(__fsub_rn(v[e], off), inv));
      uint2 pk;
      pk.x = (uint32_t)__half_as_ushort(h[0]) | ((uint32_t)__half_as_ushort(h[1]) << 16);
      pk.y = (uint32_t)__half_as_ushort(h[2]) | ((uint32_t)__half_as_ushort(h[3]) << 16);
      *(uint2*)((__half*)out + orow + x) = pk;
    } else {
      *(float4*)((float*)out + orow + x) = make_float4(v[0], v[1], v[2], v[3]);
    }
    return;
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int x = xs + j * kThreads + threadIdx.x;
    if (x >= a.W) break;
    const float rf = inv_flat(__ldg(a.flat + mrow + x), flat_norm, a.status);
    const float v = calibrate_px(__ldg(rr + x), __ldg(a.bias + mrow + x),
                                 __ldg(a.dark + mrow + x), t, rf);
    if (F16)
      ((__half*)out)[orow + x] = __float2half_rn(__fmul_rn(__fsub_rn(v, off), inv));
    else
      ((float*)out)[orow + x] = v;
  }
}

// ---------------------------------------------------------------------------
// Eight-pixel forms of the FP16 scaling sums and of calibration, for frames
// whose rows (raw, masters and outputs) start on 8-pixel boundaries.  Block b
// covers kSeg8 pixels of one row (eight consecutive pixels per thread) in
// every frame of the launch: the masters and flat_norm/flat are read and
// formed once per pixel, not once per frame, and kFrames8 frames' raw
// vectors are requested before any of them is used.
// ---------------------------------------------------------------------------
constexpr int kSeg8 = 8 * kThreads;
constexpr int kFrames8 = 4;

struct Masters8 {
  float b[8], d[8], rf[8];
};

__device__ __forceinline__ void load_masters8(const CalibArgs& a, int64_t mo, float flat_norm,
                                              Masters8& m) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const float4 b = __ldg((const float4*)(a.bias + mo) + h);
    const float4 d = __ldg((const float4*)(a.dark + mo) + h);
    const float4 f = __ldg((const float4*)(a.flat + mo) + h);
    const float bb[4] = {b.x, b.y, b.z, b.w}, dd[4] = {d.x, d.y, d.z, d.w},
                ff[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      m.b[4 * h + e] = bb[e];
      m.d[4 * h + e] = dd[e];
      m.rf[4 * h + e] = inv_flat(ff[e], flat_norm, a.status);
    }
  }
}

// The eight calibrated values of one raw vector (pixel e in the low half of
// word e / 2 for even e).
__device__ __forceinline__ void calibrate8(const uint4& q, const Masters8& m, float t,
                                           float (&v)[8]) {
  const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const float r = (e & 1) ? u16_hi_to_float(w[e >> 1]) : u16_lo_to_float(w[e >> 1]);
    v[e] = calibrate_pxf(r, m.b[e], m.d[e], t, m.rf[e]);
  }
}

// The sums that choose each frame's FP16 scaling: sum, minimum and maximum of
// the calibrated frame.  Each thread adds its eight values in FP32, the warp
// adds its 32 partials in FP32 (256 pixels), and the block's eight warp sums
// are added in FP64 and into the frame's FP64 sum.
__global__ void __launch_bounds__(kThreads) k_f16_stats8(CalibArgs a, int nk, FrameStats* st) {
  const int nseg = (a.W + kSeg8 - 1) / kSeg8;
  const int y = blockIdx.x / nseg;
  const int xs = (blockIdx.x - y * nseg) * kSeg8;
  const int x = xs + 8 * threadIdx.x;
  const bool act = x < a.W;
  const float flat_norm = a.flat_sum ? (float)(*a.flat_sum / ((double)a.W * a.H)) : 1.0f;
  Masters8 m;
  if (act) load_masters8(a, (int64_t)y * a.master_pitch + x, flat_norm, m);
  const uint16_t* rr = a.raw + (int64_t)a.k0 * a.raw_frame_stride + (int64_t)y * a.raw_pitch + x;
  const unsigned long long npx = (unsigned long long)min(kSeg8, a.W - xs);
  __shared__ float sh_sum[kThreads / 32][kFrames8];
  __shared__ int sh_min[kThreads / 32][kFrames8], sh_max[kThreads / 32][kFrames8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k0 = 0; k0 < nk; k0 += kFrames8) {
    uint4 q[kFrames8];
#pragma unroll
    for (int j = 0; j < kFrames8; ++j)
      q[j] = (act && k0 + j < nk) ? __ldg((const uint4*)(rr + (int64_t)(k0 + j) * a.raw_frame_stride))
                                  : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int j = 0; j < kFrames8; ++j) {
      float sm = 0.0f, mn = FLT_MAX, mx = -FLT_MAX;
      if (act && k0 + j < nk) {
        float v[8];
        calibrate8(q[j], m, a.t[k0 + j], v);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          sm = __fadd_rn(sm, v[e]);
          mn = fminf(mn, v[e]);
          mx = fmaxf(mx, v[e]);
        }
      }
      // the warp's 256 pixels: FP32 sum by shuffles, extremes as ordered keys
      // in one warp reduction each
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sm = __fadd_rn(sm, __shfl_xor_sync(0xffffffffu, sm, o));
      const int kmn = __reduce_min_sync(0xffffffffu, float_key(mn));
      const int kmx = __reduce_max_sync(0xffffffffu, float_key(mx));
      if (lane == 0) {
        sh_sum[warp][j] = sm;
        sh_min[warp][j] = kmn;
        sh_max[warp][j] = kmx;
      }
    }
    __syncthreads();
    if (threadIdx.x < kFrames8 && k0 + (int)threadIdx.x < nk) {
      const int j = threadIdx.x;
      double sm = 0.0;
      int kmn = INT_MAX, kmx = INT_MIN;
      for (int w = 0; w < kThreads / 32; ++w) {
        sm += (double)sh_sum[w][j];
        kmn = min(kmn, sh_min[w][j]);
        kmx = max(kmx, sh_max[w][j]);
      }
      FrameStats& f = st[a.k0 + k0 + j];
      atomicAdd(&f.sum, sm);
      atomicAdd((unsigned long long*)&f.count, npx);
      atomicMin(&f.min_key, kmn);
      atomicMax(&f.max_key, kmx);
    }
    __syncthreads();
  }
}

template <bool F16>
__global__ void __launch_bounds__(kThreads) k_calibrate8(CalibArgs a, int nk, void* out,
                                                         int64_t out_pitch, int64_t out_fstride,
                                                         const float* scale,
                                                         const float* offset) {
  const int nseg = (a.W + kSeg8 - 1) / kSeg8;
  const int y = blockIdx.x / nseg;
  const int x = (blockIdx.x - y * nseg) * kSeg8 + 8 * threadIdx.x;
  if (x >= a.W) return;
  const float flat_norm = a.flat_sum ? (float)(*a.flat_sum / ((double)a.W * a.H)) : 1.0f;
  Masters8 m;
  load_masters8(a, (int64_t)y * a.master_pitch + x, flat_norm, m);
  const uint16_t* rr = a.raw + (int64_t)a.k0 * a.raw_frame_stride + (int64_t)y * a.raw_pitch + x;
  for (int k0 = 0; k0 < nk; k0 += kFrames8) {
    uint4 q[kFrames8];
#pragma unroll
    for (int j = 0; j < kFrames8; ++j)
      if (k0 + j < nk) q[j] = __ldg((const uint4*)(rr + (int64_t)(k0 + j) * a.raw_frame_stride));
#pragma unroll
    for (int j = 0; j < kFrames8; ++j) {
      if (k0 + j >= nk) break;
      const int k = a.k0 + k0 + j;
      float v[8];
      calibrate8(q[j], m, a.t[k0 + j], v);
      const int64_t o = (int64_t)k * out_fstride + (int64_t)y * out_pitch + x;
      if (F16) {
        const float inv = __frcp_rn(__ldg(scale + k));  // exact: a power of two
        const float off = __ldg(offset + k);
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const __half lo = __float2half_rn(__fmul_rn(__fsub_rn(v[2 * e], off), inv));
          const __half hi = __float2half_rn(__fmul_rn(__fsub_rn(v[2 * e + 1], off), inv));
          w[e] = (uint32_t)__half_as_ushort(lo) | ((uint32_t)__half_as_ushort(hi) << 16);
        }
        *(uint4*)((__half*)out + o) = make_uint4(w[0], w[1], w[2], w[3]);
      } else {
        float4* po = (float4*)((float*)out + o);
        po[0] = make_float4(v[0], v[1], v[2], v[3]);
        po[1] = make_float4(v[4], v[5], v[6], v[7]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Shift, four output pixels of each of kShiftRows rows per thread (nearest,
// bilinear).  The taps of four
// neighbouring outputs overlap, so each tap of a row is read once for the
// four (five reads per row for bilinear instead of eight); taps of zero
// weight and taps only invalid outputs would use are not read.  The outputs
// (and validity bytes) leave as one vector store when vec is set and the
// four lie inside the row.  Each output is the value k_shift gives.
// ---------------------------------------------------------------------------
constexpr int kShiftRows = 4;  // output rows per thread

template <int ST, bool F16>
__global__ void __launch_bounds__(kThreads) k_shift4(ShiftArgs a, int vec) {
  const int x0 = 4 * (blockIdx.x * kThreads + threadIdx.x);
  const int kl = blockIdx.z;
  if (x0 >= a.W) return;
  const FrameDesc& F = a.frames[kl];
  const int k = a.k0 + kl;
  auto at = [&](int i, int j) -> float {
    const int64_t o = (int64_t)k * a.in_fstride + (int64_t)j * a.in_pitch + i;
    if (F16) return __half2float(__ldg((const __half*)a.in + o));
    return __ldg((const float*)a.in + o);
  };
#pragma unroll
  for (int ry = 0; ry < kShiftRows; ++ry) {
    const int y = blockIdx.y * kShiftRows + ry;
    if (y >= a.H) break;
    const bool yok = (y >= F.vy0) & (y <= F.vy1);
    bool ok[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int x = x0 + c;
      ok[c] = yok & (x >= F.vx0) & (x <= F.vx1) & (x < a.W);
    }
    const int i0 = x0 + F.ox, j0 = y + F.oy;
    float val[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) val[c] = __int_as_float(0x7fc00000);
    if (ST == ST_NEAREST) {
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (ok[c]) val[c] = at(i0 + c, j0);
    } else {
      const float fx = F.fx, fy = F.fy;
      const bool hx = fx != 0.0f, hy = fy != 0.0f;
      // column c of the taps serves output c (weight 1 - fx) and output c - 1
      // (weight fx)
      bool need[5];
      need[0] = ok[0];
#pragma unroll
      for (int c = 1; c < 4; ++c) need[c] = ok[c] || (hx && ok[c - 1]);
      need[4] = hx && ok[3];
      float r0[5], r1[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        r0[c] = need[c] ? at(i0 + c, j0) : 0.0f;
        r1[c] = (need[c] && hy) ? at(i0 + c, j0 + 1) : 0.0f;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (!ok[c]) continue;
        const float p00 = r0[c];
        const float p10 = hx ? r0[c + 1] : p00;
        const float h0 = __fmaf_rn(fx, __fsub_rn(p10, p00), p00);
        float h1 = h0;
        if (hy) {
          const float p01 = r1[c];
          const float p11 = hx ? r1[c + 1] : p01;
          h1 = __fmaf_rn(fx, __fsub_rn(p11, p01), p01);
        }
        val[c] = __fmaf_rn(fy, __fsub_rn(h1, h0), h0);
      }
    }
    const int64_t o = (int64_t)k * a.out_fstride + (int64_t)y * a.out_pitch + x0;
    if (vec && x0 + 3 < a.W) {
      if (F16) {
        const uint32_t w0 = (uint32_t)__half_as_ushort(__float2half_rn(val[0])) |
                            ((uint32_t)__half_as_ushort(__float2half_rn(val[1])) << 16);
        const uint32_t w1 = (uint32_t)__half_as_ushort(__float2half_rn(val[2])) |
                            ((uint32_t)__half_as_ushort(__float2half_rn(val[3])) << 16);
        *(uint2*)((__half*)a.out + o) = make_uint2(w0, w1);
      } else {
        *(float4*)((float*)a.out + o) = make_float4(val[0], val[1], val[2], val[3]);
      }
      if (a.valid_out)
        *(uint32_t*)(a.valid_out + o) = (ok[0] ? 1u : 0u) | (ok[1] ? 0x100u : 0u) |
                                        (ok[2] ? 0x10000u : 0u) | (ok[3] ? 0x1000000u : 0u);
      continue;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (x0 + c >= a.W) break;
      if (F16)
        ((__half*)a.out)[o + c] = __float2half_rn(val[c]);
      else
        ((float*)a.out)[o + c] = val[c];
      if (a.valid_out) a.valid_out[o + c] = ok[c] ? 1 : 0;
    }
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
      } else if (ST == ST_CUBIC) {
        // taps i0 .. i0 + 3 (origin floor(dx) - 1); with a zero fraction only
        // the second tap of the axis has non-zero weight, and only it is read
        const bool allx = F.last_tap & 1, ally = F.last_tap & 2;
        float acc = 0.0f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (!ally && q != 1) continue;
          float hh;
          if (allx) {
            hh = F.wx[0] * at(i0, j0 + q);
            hh = __fmaf_rn(F.wx[1], at(i0 + 1, j0 + q), hh);
            hh = __fmaf_rn(F.wx[2], at(i0 + 2, j0 + q), hh);
            hh = __fmaf_rn(F.wx[3], at(i0 + 3, j0 + q), hh);
          } else {
            hh = at(i0 + 1, j0 + q);
          }
          acc = ally ? (q == 0 ? F.wy[0] * hh : __fmaf_rn(F.wy[q], hh, acc)) : hh;
        }
        val = acc;
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
__device__ __forceinline__ void combine_pixel(const CombineArgs& a, float (&s)[NMAX], int x,
                                              int y, const float* s_sc, const float* s_of) {
  const float kInf = __int_as_float(0x7f800000);
  const int64_t o0 = (int64_t)y * a.pitch + x;
  // validity as one bit per frame
  uint64_t ok = ~0ull;
  if (a.valid) {
#pragma unroll
    for (int j = 0; j < NMAX; ++j)
      if (j < a.n && !__ldg(a.valid + j * a.fstride + o0)) ok &= ~(1ull << j);
  }
  int m = 0;
#pragma unroll
  for (int j = 0; j < NMAX; ++j) {
    float v = s[j];
    if (F16 && j < a.n) v = __fmaf_rn(v, s_sc[j], s_of[j]);
    v = (((ok >> j) & 1) && v == v) ? v : kInf;
    s[j] = v;
    m += (v < kInf) ? 1 : 0;
  }
  sort_network<NMAX>(s);
  const CombineOut o = combine_sorted<NMAX>(s, m, a.clip);
  const int64_t oi = (int64_t)y * a.out_pitch + x;
  if (a.mean_out) a.mean_out[oi] = o.mean;
  if (a.median_out) a.median_out[oi] = o.median;
  if (a.nkept_out) a.nkept_out[oi] = (uint16_t)o.kept;
  if (a.reject_out) {  // debug output: the samples again, in frame order
    for (int k = 0; k < a.n; ++k) {
      const int64_t ok_ = (int64_t)k * a.fstride + o0;
      float v = F16 ? __fmaf_rn(__half2float(((const __half*)a.stack)[ok_]), s_sc[k], s_of[k])
                    : __ldg((const float*)a.stack + ok_);
      if (a.valid && !a.valid[ok_]) v = kInf;
      v = (v == v) ? v : kInf;
      const bool rej = (v < kInf) & ((v < o.lo_val) | (v > o.hi_val));
      a.reject_out[((int64_t)k * a.H + y) * a.out_pitch + x] = rej ? 1 : 0;
    }
  }
}

template <int NMAX, bool F16>
__global__ void __launch_bounds__(kThreads) k_combine(CombineArgs a) {
  const int x = blockIdx.x * kThreads + threadIdx.x;
  const int y = blockIdx.y;
  __shared__ float s_sc[NMAX], s_of[NMAX];  // F16: per-frame scale and offset
  if (F16) {
    if (threadIdx.x < a.n) {
      s_sc[threadIdx.x] = a.scale[threadIdx.x];
      s_of[threadIdx.x] = a.offset[threadIdx.x];
    }
    __syncthreads();
  }
  if (x >= a.W) return;
  const float kInf = __int_as_float(0x7f800000);
  // every frame's value requested before any is used
  const int64_t o0 = (int64_t)y * a.pitch + x;
  float s[NMAX];
#pragma unroll
  for (int j = 0; j < NMAX; ++j) {
    if (j < a.n) {
      const int64_t o = (int64_t)j * a.fstride + o0;
      s[j] = F16 ? __half2float(((const __half*)a.stack)[o]) : __ldg((const float*)a.stack + o);
    } else {
      s[j] = kInf;
    }
  }
  combine_pixel<NMAX, F16>(a, s, x, y, s_sc, s_of);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_stats_init(FrameStats* st, int n, cudaStream_t s) {
  k_stats_init<<<(n + 255) / 256, 256, 0, s>>>(st, n);
  return cudaGetLastError();
}

cudaError_t launch_stats_raw(const CalibArgs& a, int nk, FrameStats* st, cudaStream_t s) {
  const int nrb = (a.H + stats_rows(a.W, a.H) - 1) / stats_rows(a.W, a.H);
  k_stats_raw<<<(unsigned)((int64_t)nk * nrb), kThreads, 0, s>>>(a, nk, st);
  return cudaGetLastError();
}

cudaError_t launch_stats_frames(const void* frames, int64_t pitch, int64_t fstride, int W, int H,
                                int n, bool f16, const float* scale, const float* offset,
                                double* sum, double* sumsq, long long* count, FrameStats* st,
                                cudaStream_t s) {
  const int nrb = (H + stats_rows(W, H) - 1) / stats_rows(W, H);
  const unsigned grid = (unsigned)((int64_t)n * nrb);
  if (f16)
    k_stats_frames<true><<<grid, kThreads, 0, s>>>(frames, pitch, fstride, W, H, n, scale, offset,
                                                   sum, sumsq, count, st);
  else
    k_stats_frames<false><<<grid, kThreads, 0, s>>>(frames, pitch, fstride, W, H, n, scale,
                                                    offset, sum, sumsq, count, st);
  return cudaGetLastError();
}

cudaError_t launch_frame_norm(const InlinePlan* inl, const void* plan_dev, int nframes,
                              int max_row_blocks, cudaStream_t s) {
  if (nframes <= 0) return cudaSuccess;
  k_frame_means<<<(unsigned)((int64_t)nframes * max_row_blocks), kThreads, 0, s>>>(*inl,
                                                                                  plan_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_frame_norm_factors<<<(nframes + 127) / 128, 128, 0, s>>>(*inl, plan_dev);
  return cudaGetLastError();
}

cudaError_t launch_f16_scaling(const FrameStats* st, int n, float* scale, float* offset,
                               cudaStream_t s) {
  k_f16_scaling<<<(n + 127) / 128, 128, 0, s>>>(st, n, scale, offset);
  return cudaGetLastError();
}

cudaError_t launch_f16_stats8(const CalibArgs& a, int nk, FrameStats* st, cudaStream_t s) {
  const int64_t grid = (int64_t)((a.W + kSeg8 - 1) / kSeg8) * a.H;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  k_f16_stats8<<<(unsigned)grid, kThreads, 0, s>>>(a, nk, st);
  return cudaGetLastError();
}

cudaError_t launch_calibrate8(const CalibArgs& a, int nk, bool f16, void* out, int64_t out_pitch,
                              int64_t out_fstride, const float* scale, const float* offset,
                              cudaStream_t s) {
  const int64_t grid = (int64_t)((a.W + kSeg8 - 1) / kSeg8) * a.H;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (f16)
    k_calibrate8<true><<<(unsigned)grid, kThreads, 0, s>>>(a, nk, out, out_pitch, out_fstride,
                                                           scale, offset);
  else
    k_calibrate8<false><<<(unsigned)grid, kThreads, 0, s>>>(a, nk, out, out_pitch, out_fstride,
                                                            scale, offset);
  return cudaGetLastError();
}

cudaError_t launch_calibrate(const CalibArgs& a, int nk, bool f16, void* out, int64_t out_pitch,
                             int64_t out_fstride, const float* scale, const float* offset,
                             cudaStream_t s) {
  const int64_t nseg = (int64_t)((a.W + kCalibSeg - 1) / kCalibSeg) * a.H;
  const int64_t grid = nseg * nk;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (f16)
    k_calibrate<true><<<(unsigned)grid, kThreads, 0, s>>>(a, nk, out, out_pitch, out_fstride,
                                                          scale, offset);
  else
    k_calibrate<false><<<(unsigned)grid, kThreads, 0, s>>>(a, nk, out, out_pitch, out_fstride,
                                                           scale, offset);
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

template <int ST>
static cudaError_t shift4_st(const ShiftArgs& a, int nk, bool f16, int vec, cudaStream_t s) {
  dim3 grid((a.W + 4 * kThreads - 1) / (4 * kThreads), (a.H + kShiftRows - 1) / kShiftRows, nk);
  if (f16)
    k_shift4<ST, true><<<grid, kThreads, 0, s>>>(a, vec);
  else
    k_shift4<ST, false><<<grid, kThreads, 0, s>>>(a, vec);
  return cudaGetLastError();
}

cudaError_t launch_shift(const ShiftArgs& a, int nk, int stencil, bool f16, int vec,
                         cudaStream_t s) {
  switch (stencil) {
    case ST_NEAREST: return shift4_st<ST_NEAREST>(a, nk, f16, vec, s);
    case ST_BILINEAR: return shift4_st<ST_BILINEAR>(a, nk, f16, vec, s);
    case ST_CUBIC: return shift_st<ST_CUBIC>(a, nk, f16, s);
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

// k_wide.cu -- combination of an aligned stack of more frames than the
// register buckets hold (Sec. 2.1 co-adding; the paper's sets reach 180
// frames per band): one CTA per 32 pixels of an output row, a group of
// lanes per pixel (wide.cuh).
#include "unfused.h"
#include "wide.cuh"

namespace irp {

// One frame's source for the CTA's output row when the samples come from
// horizontally filtered spline rows (32 bytes, shared memory).
struct RowTap {
  const float* row;  // filtered row of the first vertical tap, null if the row is invalid
  int vx0, vx1;      // valid output columns
  float wy[4];       // vertical cubic B-spline weights
  float na, nz;      // per-frame normalisation: sample = fma(sample, na, nz)
};

// The CTA gathers its [n][32] slab of samples into shared memory, then each
// of its 8 warps takes 32 / G pixels at a time, one per group of G lanes:
// load, sort (the sorted run replaces the samples in shared memory, where the
// order statistics are read), clip, and the CTA writes the results as one row.  The samples are read from an aligned stack
// (each frame's 32 pixels one 128-byte row segment), or (ROWS) formed from a
// cubic-spline frame whose rows already carry the horizontal taps: the four
// vertical taps, in the fused kernel's order, so that the samples are the same.
template <int G, int J, bool F16, bool ROWS>
__global__ void __launch_bounds__(kWideThreads) k_combine_wide(CombineArgs a, int tiles_x) {
  extern __shared__ float s_wide[];
  __shared__ float s_mean[32], s_median[32];
  __shared__ int s_kept[32];
  using SM = WideSmem<G, J>;
  constexpr int P = 32 / G;  // pixels per warp at a time
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
  if (ROWS) {
    // the frames' sources for this output row, after the sample slab
    RowTap* tab = (RowTap*)(s_wide + SM::kBytes / sizeof(float));
    for (int k = t; k < n; k += kWideThreads) {
      const FrameDesc* F = a.frames + k;
      RowTap r;
      const int vy0 = __ldg(&F->vy0), vy1 = __ldg(&F->vy1);
      const float* coef = (const float*)__ldg((const unsigned long long*)&F->coef);
      r.row = (y >= vy0 && y <= vy1) ? coef + (int64_t)(y + __ldg(&F->oy) + 2) * a.coef_pitch
                                     : nullptr;
      r.vx0 = __ldg(&F->vx0);
      r.vx1 = __ldg(&F->vx1);
#pragma unroll
      for (int j = 0; j < 4; ++j) r.wy[j] = __ldg(&F->wy[j]);
      const FrameNorm* nr = (const FrameNorm*)__ldg((const unsigned long long*)&F->norm);
      r.na = nr ? nr->na : 1.0f;
      r.nz = nr ? nr->nz : 0.0f;
      tab[k] = r;
    }
    __syncthreads();
    const int x = x0 + lane;
    const int64_t p1 = a.coef_pitch;
    constexpr int kBatch = 4;  // samples (4 loads each) in flight per thread
    for (int k0 = warp; k0 < n; k0 += 8 * kBatch) {
      float h[kBatch][4];
      float4 w[kBatch];
#pragma unroll
      for (int b = 0; b < kBatch; ++b) {
        const int k = k0 + 8 * b;
        const RowTap r =
            k < n ? tab[k] : RowTap{nullptr, 0, -1, {0.0f, 0.0f, 0.0f, 0.0f}, 1.0f, 0.0f};
        const bool ok = r.row && x >= r.vx0 && x <= r.vx1;
        w[b] = make_float4(r.wy[0], r.wy[1], r.wy[2], r.wy[3]);
#pragma unroll
        for (int j = 0; j < 4; ++j) h[b][j] = ok ? __ldg(r.row + x + j * p1) : kInf;
      }
#pragma unroll
      for (int b = 0; b < kBatch; ++b) {
        const int k = k0 + 8 * b;
        if (k >= n) continue;
        float acc = w[b].x * h[b][0];
        acc = __fmaf_rn(w[b].y, h[b][1], acc);
        acc = __fmaf_rn(w[b].z, h[b][2], acc);
        acc = __fmaf_rn(w[b].w, h[b][3], acc);
        if (a.frame_norm) acc = __fmaf_rn(acc, tab[k].na, tab[k].nz);
        s_wide[SM::at(lane, k)] = h[b][0] < kInf ? acc : kInf;
      }
    }
  } else {
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
  const int g = lane / G, tg = lane % G;  // the lane's group and its index in it
#pragma unroll 1
  for (int q = warp; q < 32 / P; q += 8) {
    // the warp's groups take pixels 32 / P apart (conflict-free shared memory);
    // pixels past the frame were staged as invalid and give no output
    const int p = q + g * (32 / P);
    float* const col = s_wide + SM::at(p, 0);  // this pixel's samples
    float v[J];
    int cnt = 0;
#pragma unroll
    for (int i = 0; i < J; ++i) {
      const int e = tg * J + i;
      v[i] = e < n ? col[tg * (J + 1) + i] : kInf;
      cnt += v[i] < kInf ? 1 : 0;
    }
    const int m = group_sum_i<G>(cnt);
    group_bitonic_sort<G, J>(v, tg);
    // the sorted run replaces the pixel's samples (sample e at col[e + e / J])
    __syncwarp();
#pragma unroll
    for (int i = 0; i < J; ++i) col[tg * (J + 1) + i] = v[i];
    __syncwarp();
    const WideOut o = group_combine<G, J>(v, col, m, a.clip, tg);
    if (tg == 0) {
      s_mean[p] = o.mean;
      s_median[p] = o.median;
      s_kept[p] = o.kept;
    }
    const int x = x0 + p;
    if (!ROWS && a.reject_out && x < a.W) {  // debug output: the samples again, in frame order
      const int64_t o0 = (int64_t)y * a.pitch + x;
      for (int k = tg; k < n; k += G) {
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

template <int G, int J, bool F16, bool ROWS>
static cudaError_t combine_wide_j(const CombineArgs& a, cudaStream_t s) {
  static size_t granted = 0;
  const size_t smem = WideSmem<G, J>::kBytes + (ROWS ? (size_t)a.n * sizeof(RowTap) : 0);
  auto fn = k_combine_wide<G, J, F16, ROWS>;
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

template <bool F16, bool ROWS>
static cudaError_t combine_wide_f(const CombineArgs& a, cudaStream_t s) {
  static_assert(wide_j(1) == 32, "one sample count per lane");
  switch (wide_g(a.n)) {
    case 4: return combine_wide_j<4, 32, F16, ROWS>(a, s);
    case 8: return combine_wide_j<8, 32, F16, ROWS>(a, s);
    case 16: return combine_wide_j<16, 32, F16, ROWS>(a, s);
    default: return combine_wide_j<32, 32, F16, ROWS>(a, s);
  }
}

cudaError_t launch_combine_wide(const CombineArgs& a, bool f16, cudaStream_t s) {
  if (a.n < 1 || a.n > kWideMaxFrames) return cudaErrorInvalidValue;
  if (!a.stack) return a.frames ? combine_wide_f<false, true>(a, s) : cudaErrorInvalidValue;
  return f16 ? combine_wide_f<true, false>(a, s) : combine_wide_f<false, false>(a, s);
}

}  // namespace irp

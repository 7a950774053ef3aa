// k_spline.cu -- cubic-spline coefficients of calibrated raw frames, row pass
// and column pass without tile halos.
//
// Sec. 3.2.1: one tridiagonal system per row and per column.  As in
// prefilter.cuh the mirror-boundary solution is c = sqrt(3)(y+ + y- - v) with
// y+[i] = v[i] + z1 y+[i-1] and y-[i] = v[i] + z1 y-[i+1], z1 = sqrt(3) - 2.
//
// Row pass: one CTA per frame row and chunk of kRowGroup = 16 frames; the
// row's masters and 1/flat are staged in shared memory once for the chunk,
// and each warp reduces two frames of the row (both rows loaded up front).  Lane l calibrates and holds the E
// columns [E l, E l + E) in registers and runs both recursions over them from
// zero; the value entering from the neighbouring lane is added afterwards,
// y+[E l + j] = local+[j] + z1^(j+1) y+[E l - 1] (and likewise for y-), which
// is exact up to z1^E (< 5e-19 for E >= 32).  The mirror boundary is exact:
// y+[-1] is the sum of z1^k v[1+k], and y-[W-1] = y+[W-1].
//
// Column pass: one thread per (frame, column, 32-row segment), coalesced
// across the warp's columns, warm-up of 16 rows on each side read from the
// mirror-extended rows; the result is written into the padded coefficient
// frame together with its 2-sample mirrored border.
#include "prefilter.cuh"
#include "reduce_kernels.cuh"
#include "spline.h"

namespace irp {

namespace {

template <int E>
struct ZPow {  // z1^1 .. z1^E
  float p[E + 1];
  __host__ __device__ constexpr ZPow() : p() {
    double z = -0.26794919243112270, a = 1.0;
    for (int i = 0; i <= E; ++i) {
      p[i] = (float)a;
      a *= z;
    }
  }
};

__device__ __forceinline__ int find_by(const SetDesc* sets, int nsets, int item, int which) {
  int lo = 0, hi = nsets - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int p = which == 0 ? sets[mid].row0 : sets[mid].colseg0;
    if (p <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace

template <int E>
__global__ void __launch_bounds__(256, 2)
    k_spline_rows(const __grid_constant__ InlinePlan inl, const void* plan_dev) {
  // masters of the block's row, element x at [x % E][x / E] (stride 33): lane
  // l reads column E l + j from word j*33 + l, one bank per lane
  __shared__ float sm[3][E * 33];
  const PlanView P = make_view(inl, plan_dev);
  const int item = blockIdx.x;
  if (item >= P.h->nrows) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const SetDesc& S = P.sets[find_by(P.sets, P.h->nsets, item, 0)];
  const int local = item - S.row0;
  const int g = local / S.H, y = local - g * S.H;  // frame chunk, row
  const int W = S.W;
  const int x0 = lane * E;
  {
    const float flat_norm = S.flat_sum ? (float)(*S.flat_sum / ((double)W * S.H)) : 1.0f;
    const int64_t mo = (int64_t)y * S.master_pitch;
    for (int x = threadIdx.x; x < 32 * E; x += 256) {
      const int si = (x % E) * 33 + x / E;
      if (x < W) {
        sm[0][si] = __ldg(S.bias + mo + x);
        sm[1][si] = __ldg(S.dark + mo + x);
        sm[2][si] = inv_flat(__ldg(S.flat + mo + x), flat_norm, P.h->status);
      } else {
        sm[0][si] = sm[1][si] = sm[2][si] = 0.0f;
      }
    }
  }
  __syncthreads();
  constexpr ZPow<E> zp{};
  // each warp reduces frames k and k + 8 of the chunk; both raw rows are
  // requested before the first is used
  constexpr int kQ = E / 8;  // 16-byte raw loads per lane and row
  uint4 q[2][kQ];
  int kf[2] = {g * kRowGroup + warp, g * kRowGroup + warp + 8};
#pragma unroll
  for (int f = 0; f < 2; ++f) {
    if (kf[f] < S.n) {
      const FrameDesc& F = P.frames[S.frame0 + kf[f]];
      const uint16_t* raw = (const uint16_t*)F.src + (int64_t)y * S.src_pitch;
      if ((F.flags & 1) && x0 + E <= W) {
#pragma unroll
        for (int i = 0; i < kQ; ++i) q[f][i] = __ldg((const uint4*)(raw + x0) + i);
      }
    }
  }
#pragma unroll 1
  for (int f = 0; f < 2; ++f) {
    const int k = kf[f];
    if (k >= S.n) break;
    const FrameDesc& F = P.frames[S.frame0 + k];
    const uint16_t* raw = (const uint16_t*)F.src + (int64_t)y * S.src_pitch;
    const float t = F.t;
    float v[E];
    if ((F.flags & 1) && x0 + E <= W) {
#pragma unroll
      for (int j = 0; j < E; j += 8) {
        const uint4 qq = f == 0 ? q[0][j / 8] : q[1][j / 8];
        const uint32_t w[4] = {qq.x, qq.y, qq.z, qq.w};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int si = (j + i) * 33 + lane;
          v[j + i] = calibrate_px((uint16_t)(w[i >> 1] >> (16 * (i & 1))), sm[0][si], sm[1][si],
                                  t, sm[2][si]);
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const int si = j * 33 + lane;
        v[j] = x0 + j < W ? calibrate_px(__ldg(raw + x0 + j), sm[0][si], sm[1][si], t, sm[2][si])
                          : 0.0f;
      }
    }
    // causal recursion within the lane, then the carry from the left lane
    float yp[E];
    {
      float acc = 0.0f;
#pragma unroll
      for (int j = 0; j < E; ++j) {
        acc = __fmaf_rn(kZ1, acc, v[j]);
        yp[j] = acc;
      }
      float carry = __shfl_up_sync(0xffffffffu, yp[E - 1], 1);
      if (lane == 0) {  // y+[-1] = sum_k z1^k v[1+k] (mirror)
        float m = 0.0f;
#pragma unroll
        for (int j = E - 1; j >= 1; --j) m = __fmaf_rn(kZ1, m, v[j]);
        carry = m;
      }
#pragma unroll
      for (int j = 0; j < E; ++j) yp[j] = __fmaf_rn(zp.p[j + 1], carry, yp[j]);
    }
    // anti-causal recursion: starts at W-1 with y-[W-1] = y+[W-1] (mirror).  A
    // first pass over the lane finds its local value at the left end, the carry
    // into the left neighbour; the second pass starts from the carry of the
    // right neighbour and emits the coefficients.
    float carry;
    {
      float acc = 0.0f;
#pragma unroll
      for (int j = E - 1; j >= 0; --j) {
        const int x = x0 + j;
        acc = x > W - 1 ? 0.0f : (x == W - 1 ? yp[j] : __fmaf_rn(kZ1, acc, v[j]));
      }
      carry = __shfl_down_sync(0xffffffffu, acc, 1);
      if (x0 + E - 1 >= W - 1) carry = 0.0f;
    }
    float* out = F.crow + (int64_t)y * S.crow_pitch + x0;
    const bool vst = x0 + E <= W && (S.crow_pitch & 3) == 0;
    float acc = carry;
    float c4[4];
#pragma unroll
    for (int j = E - 1; j >= 0; --j) {
      const int x = x0 + j;
      acc = x > W - 1 ? 0.0f : (x == W - 1 ? yp[j] : __fmaf_rn(kZ1, acc, v[j]));
      const float c = __fmul_rn(kSqrt3, __fsub_rn(__fadd_rn(yp[j], acc), v[j]));
      if (vst) {
        c4[j & 3] = c;
        if ((j & 3) == 0) *(float4*)(out + j) = make_float4(c4[0], c4[1], c4[2], c4[3]);
      } else if (x < W) {
        out[j] = c;
      }
    }
  }
}

constexpr int kColSeg = 32;  // output rows per column task

__global__ void __launch_bounds__(256, 2)
    k_spline_cols(const __grid_constant__ InlinePlan inl, const void* plan_dev) {
  const PlanView P = make_view(inl, plan_dev);
  const int item = blockIdx.x * 256 + threadIdx.x;
  if (item >= P.h->ncolsegs) return;
  const SetDesc& S = P.sets[find_by(P.sets, P.h->nsets, item, 1)];
  const int W = S.W, H = S.H;
  const int nseg = (H + kColSeg - 1) / kColSeg;
  const int local = item - S.colseg0;
  const int k = local / (W * nseg);
  const int rem = local - k * (W * nseg);
  const int seg = rem / W, x = rem - seg * W;
  const FrameDesc& F = P.frames[S.frame0 + k];
  const float* in = F.crow + x;
  const int64_t ip = S.crow_pitch;
  const int y0 = seg * kColSeg;
  constexpr int L = kColSeg + 2 * kPrefHalo;
  float v[L];
  const bool inner = y0 - kPrefHalo >= 0 && y0 + kColSeg + kPrefHalo <= H;
  if (inner) {
    const float* p = in + (int64_t)(y0 - kPrefHalo) * ip;
#pragma unroll
    for (int j = 0; j < L; ++j) v[j] = __ldg(p + (int64_t)j * ip);
  } else {
#pragma unroll
    for (int j = 0; j < L; ++j) {
      int yy = y0 - kPrefHalo + j;  // one reflection suffices: H >= kSplineMinSide > kPrefHalo
      yy = yy < 0 ? -yy : (yy >= H ? 2 * H - 2 - yy : yy);
      v[j] = __ldg(in + (int64_t)yy * ip);
    }
  }
  float yp[kColSeg];
  float acc = 0.0f;
#pragma unroll
  for (int j = 0; j < kPrefHalo; ++j) acc = __fmaf_rn(kZ1, acc, v[j]);
#pragma unroll
  for (int j = 0; j < kColSeg; ++j) {
    acc = __fmaf_rn(kZ1, acc, v[kPrefHalo + j]);
    yp[j] = acc;
  }
  acc = 0.0f;
#pragma unroll
  for (int j = L - 1; j >= kPrefHalo + kColSeg; --j) acc = __fmaf_rn(kZ1, acc, v[j]);
  // padded frame (x, y) at (y + 2) * pitch + x + 2; the 2-sample border
  // holds the mirrored coefficients: c[-1] = c[1], c[-2] = c[2],
  // c[W] = c[W-2], c[W+1] = c[W-3] (likewise for rows)
  float* out = F.coef;
  const int64_t cp = S.coef_pitch;
  const int bx1 = x == 1 ? -1 : (x == W - 2 ? W : -100);
  const int bx2 = x == 2 ? -2 : (x == W - 3 ? W + 1 : -100);
  const bool xedge = bx1 != -100 || bx2 != -100;
  const bool yedge = y0 < 3 || y0 + kColSeg > H - 3;
  if (!xedge && !yedge && y0 + kColSeg <= H) {
    float* o = out + (int64_t)(y0 + kColSeg - 1 + 2) * cp + (x + 2);
#pragma unroll
    for (int j = kColSeg - 1; j >= 0; --j) {
      const float vj = v[kPrefHalo + j];
      acc = __fmaf_rn(kZ1, acc, vj);
      *o = __fmul_rn(kSqrt3, __fsub_rn(__fadd_rn(yp[j], acc), vj));
      o -= cp;
    }
    return;
  }
#pragma unroll
  for (int j = kColSeg - 1; j >= 0; --j) {
    const float vj = v[kPrefHalo + j];
    acc = __fmaf_rn(kZ1, acc, vj);
    const int y = y0 + j;
    if (y >= H) continue;
    const float c = __fmul_rn(kSqrt3, __fsub_rn(__fadd_rn(yp[j], acc), vj));
    out[(int64_t)(y + 2) * cp + (x + 2)] = c;
    const int by1 = y == 1 ? -1 : (y == H - 2 ? H : -100);
    const int by2 = y == 2 ? -2 : (y == H - 3 ? H + 1 : -100);
    if (xedge || by1 != -100 || by2 != -100) {
      const int ys[3] = {y, by1, by2}, xs[3] = {x, bx1, bx2};
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
          if ((a | b) && ys[a] != -100 && xs[b] != -100)
            out[(int64_t)(ys[a] + 2) * cp + (xs[b] + 2)] = c;
    }
  }
}

cudaError_t launch_spline_rows(int e, const InlinePlan* inl, const void* plan_dev, int nrows,
                               cudaStream_t s) {  // nrows: (row, frame group) work items
  const int grid = nrows;
  if (e == 32)
    k_spline_rows<32><<<grid, 256, 0, s>>>(*inl, plan_dev);
  else
    k_spline_rows<64><<<grid, 256, 0, s>>>(*inl, plan_dev);
  return cudaGetLastError();
}

cudaError_t launch_spline_cols(const InlinePlan* inl, const void* plan_dev, int ncolsegs,
                               cudaStream_t s) {
  k_spline_cols<<<(ncolsegs + 255) / 256, 256, 0, s>>>(*inl, plan_dev);
  return cudaGetLastError();
}

}  // namespace irp

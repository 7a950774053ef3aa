// k_spline.cu -- cubic-spline coefficients of calibrated raw frames, row pass
// and column pass without tile halos; the column pass also applies the
// horizontal taps of each frame's resampling.
//
// Sec. 3.2.1: one tridiagonal system per row and per column.  As in
// prefilter.cuh the mirror-boundary solution is c = sqrt(3)(y+ + y- - v) with
// y+[i] = v[i] + z1 y+[i-1] and y-[i] = v[i] + z1 y-[i+1], z1 = sqrt(3) - 2.
//
// Row pass: one CTA per block of rows (4, or 2 for frames wider than 1024)
// and chunk of at most kRowGroup frames.  The block's master rows are copied into
// shared memory asynchronously and 1/flat is formed in place; the warps take
// the block's (row, frame) tasks round-robin and prefetch the next task's raw
// row with cp.async while computing the current one.  Lane l calibrates and
// holds the E columns [E l, E l + E) in registers and runs both recursions
// over them from zero; the value entering from the neighbouring lane is added
// afterwards, y+[E l + j] = local+[j] + z1^(j+1) y+[E l - 1] (and likewise for
// y-), which is exact up to z1^E (< 5e-19 for E >= 32).  The mirror boundary
// is exact: y+[-1] is the sum of z1^k v[1+k], and y-[W-1] = y+[W-1].
//
// Column pass: one CTA per (frame, 29 output columns, kColRows rows); lane =
// column, warp = 32 consecutive rows.  Lane l solves the source column the
// frame's first horizontal tap of output column l falls on.  Each warp runs
// both recursions over its rows from zero, the warps exchange their ends
// through shared memory (the carry from the warp above / below, exact up to
// z1^32), and the CTA's first and last warp take their outer carry from 16
// warm-up rows of the mirror-extended column.  The coefficients then take the
// frame's 4 horizontal B-spline taps from lanes l .. l + 3, so the frame
// written is the coefficients filtered along x on the output grid, with a
// 2-row mirrored border: the fused kernel only applies the vertical taps.
#include <algorithm>

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
    k_spline_rows(const __grid_constant__ InlinePlan inl, const void* plan_dev, int item0,
                  int stride) {
  constexpr int RB = row_block(E);   // rows per CTA
  constexpr int MQ = E / 4;          // float4 master chunks per lane and row
  constexpr int RQ = E / 8;          // 16-byte raw chunks per lane and row
  extern __shared__ __align__(16) float4 smem4[];
  // masters: [row][bias, dark, rf][MQ][32 lanes] float4 (lane l holds columns
  // E l .. E l + E - 1, chunk i = columns E l + 4i .. + 3): conflict-free
  float4* s_m = smem4;
  // raw: per warp kRowStages stages of [RQ][32 lanes] uint4
  uint4* s_raw = (uint4*)(smem4 + RB * 3 * MQ * 32);
  // E = 32: per-warp output row, chunk c = 8 l + i of lane l at 8 l + (i ^ (l & 7))
  // (conflict-free for the lane-wise writes and the row-order reads)
  float4* s_out = (float4*)(s_raw + 8 * kRowStages * RQ * 32) + (threadIdx.x >> 5) * 256;
  const PlanView P = make_view(inl, plan_dev);
  const int item = item0 + (int)blockIdx.x * stride;
  if (item >= P.h->nrows) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const SetDesc& S = P.sets[find_by(P.sets, P.h->nsets, item, 0)];
  if (S.ready_flag) {  // the set's raw frames may still be arriving
    __shared__ int s_ok;
    if (threadIdx.x == 0)
      s_ok = wait_ready(S.ready_flag, S.ready_value, P.h->spin_limit, P.h->status);
    __syncthreads();
    if (!s_ok) return;  // status latched
  }
  const int H = S.H;
  // row block major, so that a range of row blocks is a range of work items;
  // within a row block, segment major
  const int rg = S.rgroup;
  const int ngroups = (S.n + rg - 1) / rg;
  const int nseg = row_segments(S.W);
  const int local = item - S.row0;
  const int rb = local / (ngroups * nseg);
  const int rem = local - rb * (ngroups * nseg);
  const int sg = rem / ngroups, g = rem - sg * ngroups;  // segment, frame chunk
  // this item's columns: source [xs, xs + W) of the row, coefficients kept
  // for the core [c0, c1) (relative: [cl, cr))
  int c0, c1, xs;
  row_segment(S.W, sg, c0, c1, xs);
  const int W = min(S.W - xs, kSegCols);
  const int cl = c0 - xs, cr = c1 - xs;
  const int y0 = rb * RB, nr = min(RB, H - y0);
  const int k0 = g * rg, nk = min(rg, S.n - k0);
  const int x0 = lane * E;
  // 1. the block's master rows, asynchronously (zero beyond the frame)
  {
    const bool vec = S.mflags & 1;
    if (vec) {
      for (int c = threadIdx.x; c < RB * 3 * 8 * E; c += 256) {  // 16-byte chunks
        const int rr = c / (3 * 8 * E), rem = c - rr * (3 * 8 * E);
        const int a = rem / (8 * E), xc = rem - a * (8 * E);   // chunk xc: columns 4xc..
        const int x = 4 * xc, l = x / E, i = (x - l * E) >> 2;
        const int y = y0 + rr;
        const int nb = (rr < nr && x < W) ? 4 * min(4, W - x) : 0;
        const float* base = a == 0 ? S.bias : (a == 1 ? S.dark : S.flat);
        const float* gp = nb ? base + (int64_t)y * S.master_pitch + xs + x : S.bias;
        cp_async16(s_m + ((rr * 3 + a) * MQ + i) * 32 + l, gp, nb);
      }
    } else {
      for (int c = threadIdx.x; c < RB * 3 * 32 * E; c += 256) {  // single floats
        const int rr = c / (3 * 32 * E), rem = c - rr * (3 * 32 * E);
        const int a = rem / (32 * E), x = rem - a * (32 * E);
        const int l = x / E, j = x - l * E;
        const int y = y0 + rr;
        const int nb = (rr < nr && x < W) ? 4 : 0;
        const float* base = a == 0 ? S.bias : (a == 1 ? S.dark : S.flat);
        const float* gp = nb ? base + (int64_t)y * S.master_pitch + xs + x : S.bias;
        cp_async4((float*)(s_m + ((rr * 3 + a) * MQ + (j >> 2)) * 32 + l) + (j & 3), gp, nb);
      }
    }
    cp_async_commit();
  }
  // the chunk's frame fields, read once per CTA instead of once per task
  __shared__ const uint16_t* s_src[kRowGroup];
  __shared__ float* s_crow[kRowGroup];
  __shared__ float s_t[kRowGroup];
  __shared__ int s_flags[kRowGroup];
  __shared__ uint32_t* s_bad[kRowGroup];
  if (threadIdx.x < nk) {
    const FrameDesc& F = P.frames[S.frame0 + k0 + threadIdx.x];
    s_src[threadIdx.x] = (const uint16_t*)F.src;
    s_crow[threadIdx.x] = F.crow;
    s_t[threadIdx.x] = F.t;
    s_flags[threadIdx.x] = F.flags;
    s_bad[threadIdx.x] = const_cast<uint32_t*>(F.bad);
  }
  const bool masked = S.masked != 0;
  __syncthreads();
  // 2. the warp's tasks: (row, frame) pairs of the block, t = warp + 8 m
  const int ntask = nr * nk;
  uint4* stage = s_raw + warp * kRowStages * RQ * 32;
  // the row's 16-byte chunks in order (contiguous per instruction), each put
  // where its owner lane reads it: chunk c of lane c / RQ at (c % RQ) * 32 + c / RQ.
  // Rows 16-byte aligned take one copy per chunk, rows 8-byte aligned (pitch
  // 4k, e.g. 1020 columns) two; the columns past the row are zero-filled.
  auto issue = [&](int t, int slot) {
    const int rr = t / nk, f = t - rr * nk;
    const int fl = s_flags[f];
    const uint16_t* raw = s_src[f] + (int64_t)(y0 + rr) * S.src_pitch + xs;
#pragma unroll
    for (int k = 0; k < RQ; ++k) {
      const int c = 32 * k + lane, lc = c / RQ, ic = c - lc * RQ;
      const int nb = max(0, min(16, 2 * (W - 8 * c)));  // bytes inside the row
      uint4* dst = stage + (slot * RQ + ic) * 32 + lc;
      if (fl & 1) {
        cp_async16(dst, nb ? raw + 8 * c : raw, nb);
      } else if (fl & 2) {
        cp_async8(dst, nb ? raw + 8 * c : raw, min(nb, 8));
        cp_async8((uint8_t*)dst + 8, nb > 8 ? raw + 8 * c + 4 : raw, max(nb - 8, 0));
      }
    }
  };
#pragma unroll
  for (int q = 0; q < kRowStages - 1; ++q) {
    if (warp + 8 * q < ntask) issue(warp + 8 * q, q);
    cp_async_commit();
  }
  // 3. masters landed: flat -> flat_norm / flat in place
  cp_async_wait<kRowStages - 1>();
  __syncthreads();
  {
    const float flat_norm = S.flat_sum ? (float)(*S.flat_sum / ((double)S.W * H)) : 1.0f;
    for (int c = threadIdx.x; c < RB * MQ * 32; c += 256) {
      const int rr = c / (MQ * 32), rem = c - rr * (MQ * 32);
      const int i = rem >> 5, l = rem & 31;
      float* q = (float*)(s_m + ((rr * 3 + 2) * MQ + i) * 32 + l);
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (rr < nr && l * E + 4 * i + e < W) q[e] = inv_flat(q[e], flat_norm, P.h->status);
    }
  }
  __syncthreads();
  constexpr ZPow<E> zp{};
  int m = 0;
#pragma unroll 1
  for (int t = warp; t < ntask; t += 8, ++m) {
    if (t + 8 * (kRowStages - 1) < ntask) issue(t + 8 * (kRowStages - 1), (m + kRowStages - 1) % kRowStages);
    cp_async_commit();
    cp_async_wait<kRowStages - 1>();
    __syncwarp();
    const int rr = t / nk, f = t - rr * nk;
    const int y = y0 + rr;
    const float tk = s_t[f];
    const bool vec = (s_flags[f] & 3) != 0;  // staged (zero past the row)
    const float4* mb = s_m + (rr * 3 + 0) * MQ * 32 + lane;
    const float4* md = mb + MQ * 32;
    const float4* mr = md + MQ * 32;
    float v[E];
    if (vec) {
      const uint4* rs = stage + ((m % kRowStages) * RQ) * 32 + lane;
#pragma unroll
      for (int i = 0; i < RQ; ++i) {
        const uint4 qq = rs[i * 32];
        const uint32_t w[4] = {qq.x, qq.y, qq.z, qq.w};
        const float4 b0 = mb[(2 * i) * 32], b1 = mb[(2 * i + 1) * 32];
        const float4 d0 = md[(2 * i) * 32], d1 = md[(2 * i + 1) * 32];
        const float4 r0 = mr[(2 * i) * 32], r1 = mr[(2 * i + 1) * 32];
        const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
        const float dd[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
        const float rf[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
#pragma unroll
        for (int e = 0; e < 8; ++e)
          v[8 * i + e] = calibrate_pxf((e & 1) ? u16_hi_to_float(w[e >> 1])
                                               : u16_lo_to_float(w[e >> 1]),
                                       bb[e], dd[e], tk, rf[e]);
      }
    } else {
      const uint16_t* raw = s_src[f] + (int64_t)y * S.src_pitch + xs;
#pragma unroll
      for (int i = 0; i < MQ; ++i) {
        const float4 b = mb[i * 32], d = md[i * 32], r = mr[i * 32];
        const float bb[4] = {b.x, b.y, b.z, b.w}, dd[4] = {d.x, d.y, d.z, d.w};
        const float rf[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int x = x0 + 4 * i + e;
          v[4 * i + e] = x < W ? calibrate_px(__ldg(raw + x), bb[e], dd[e], tk, rf[e]) : 0.0f;
        }
      }
    }
    if (masked) {
      // this row's bad pixels (marked by the mask master, or raw at the
      // saturation level) as bits, 32 columns per word, for the tile kernel
      const uint8_t* mrow = S.mask ? S.mask + (int64_t)y * S.mask_pitch + xs : nullptr;
      const uint16_t* rrow = s_src[f] + (int64_t)y * S.src_pitch + xs;
      uint32_t* brow = s_bad[f] + (int64_t)y * S.bad_pitch + (xs >> 5);
#pragma unroll
      for (int wd = 0; wd < E / 32; ++wd) {
        uint32_t bits = 0;
#pragma unroll 1
        for (int e = 0; e < 32; ++e) {
          const int x = x0 + 32 * wd + e;
          if (x < W && ((float)__ldg(rrow + x) >= S.saturation || (mrow && __ldg(mrow + x))))
            bits |= 1u << e;
        }
        if (x0 + 32 * wd < W) brow[(x0 >> 5) + wd] = bits;
      }
    }
    // causal recursion within the lane, as two independent half-lane chains
    // joined exactly (y+[h + j] gets z1^(j+1) y+[h - 1]), then the carry
    // from the left lane
    constexpr int Hh = E / 2;
    float yp[E];
    {
      float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
      for (int j = 0; j < Hh; ++j) {
        a0 = __fmaf_rn(kZ1, a0, v[j]);
        a1 = __fmaf_rn(kZ1, a1, v[Hh + j]);
        yp[j] = a0;
        yp[Hh + j] = a1;
      }
#pragma unroll
      for (int j = 0; j < Hh; ++j) yp[Hh + j] = __fmaf_rn(zp.p[j + 1], a0, yp[Hh + j]);
      float carry = __shfl_up_sync(0xffffffffu, yp[E - 1], 1);
      if (lane == 0) {  // y+[-1] = sum_k z1^k v[1+k] (mirror), as two chains
        float lo = 0.0f, hi = 0.0f;
#pragma unroll
        for (int j = Hh - 1; j >= 1; --j) lo = __fmaf_rn(kZ1, lo, v[j]);
#pragma unroll
        for (int j = E - 1; j >= Hh; --j) hi = __fmaf_rn(kZ1, hi, v[j]);
        carry = __fmaf_rn(zp.p[Hh - 1], hi, lo);
      }
#pragma unroll
      for (int j = 0; j < E; ++j) yp[j] = __fmaf_rn(zp.p[j + 1], carry, yp[j]);
    }
    float* out = s_crow[f] + (int64_t)y * S.crow_pitch + xs + x0;
    if (W % E == 0) {
      // the frame ends at the end of lane `last`: y-[W-1] = y+[W-1] is set at a
      // fixed position, and the lanes past it (zeros) pass no carry
      const int last = W / E - 1;
      const bool is_last = lane == last;
      // the lane's value at its left end, as two half-lane chains
      float hi = is_last ? yp[E - 1] : v[E - 1], lo = 0.0f;
#pragma unroll
      for (int t = 1; t < Hh; ++t) hi = __fmaf_rn(kZ1, hi, v[E - 1 - t]);
#pragma unroll
      for (int j = Hh - 1; j >= 0; --j) lo = __fmaf_rn(kZ1, lo, v[j]);
      float carry = __shfl_down_sync(0xffffffffu, __fmaf_rn(zp.p[Hh], hi, lo), 1);
      if (lane >= last) carry = 0.0f;
      // the lane's coefficients go to the row buffer (E = 32) or straight out
      auto put = [&](int j, float4 c) {
        if (E == 32)
          s_out[8 * lane + ((j >> 2) ^ (lane & 7))] = c;
        else if (x0 + j >= cl && x0 + j < cr)  // the segment's core (4 | cl, cr)
          *(float4*)(out + j) = c;
      };
      if (lane <= last) {
        // upper half from the carry (emitting its coefficients) and lower half
        // from zero, side by side; then the lower half gets z1^(h-j) y-[h]
        float ah = carry, al = 0.0f, ml[Hh];
        float c4[4];
#pragma unroll
        for (int t = 0; t < Hh; ++t) {
          const int j = E - 1 - t;
          ah = (j == E - 1 && is_last) ? yp[j] : __fmaf_rn(kZ1, ah, v[j]);
          al = __fmaf_rn(kZ1, al, v[Hh - 1 - t]);
          ml[Hh - 1 - t] = al;
          c4[j & 3] = __fmul_rn(kSqrt3, __fsub_rn(__fadd_rn(yp[j], ah), v[j]));
          if ((j & 3) == 0) put(j, make_float4(c4[0], c4[1], c4[2], c4[3]));
        }
#pragma unroll
        for (int j = Hh - 1; j >= 0; --j) {
          const float m = __fmaf_rn(zp.p[Hh - j], ah, ml[j]);
          c4[j & 3] = __fmul_rn(kSqrt3, __fsub_rn(__fadd_rn(yp[j], m), v[j]));
          if ((j & 3) == 0) put(j, make_float4(c4[0], c4[1], c4[2], c4[3]));
        }
      }
      if (E == 32) {
        // the row in order: chunk g = 32 k + lane, contiguous per instruction
        __syncwarp();
        float* row = s_crow[f] + (int64_t)y * S.crow_pitch;
        const int nchunk = W / 4;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int g = 32 * k + lane;
          const int l = g >> 3, i = g & 7;
          if (g < nchunk) *(float4*)(row + 4 * g) = s_out[8 * l + (i ^ (l & 7))];
        }
        __syncwarp();
      }
    } else {
      // anti-causal recursion: starts at W-1 with y-[W-1] = y+[W-1] (mirror).
      // A first pass over the lane finds its local value at the left end, the
      // carry into the left neighbour; the second pass starts from the carry
      // of the right neighbour and emits the coefficients.
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
          if ((j & 3) == 0 && x >= cl && x < cr)
            *(float4*)(out + j) = make_float4(c4[0], c4[1], c4[2], c4[3]);
        } else if (x >= cl && x < cr) {
          out[j] = c;
        }
      }
    }
    __syncwarp();  // this stage is refilled kRowStages tasks later
  }
  cp_async_wait<0>();
}


constexpr int kColWarps = kColRows / 32;  // one warp per 32 rows
constexpr int kColWarm = 16;   // warm-up rows above and below the CTA's rows
constexpr int kColOut = 29;    // output columns per CTA: lanes 0..28 (taps reach lane + 3)

__global__ void __launch_bounds__(kColRows, kColRows < 512 ? 512 / kColRows : 1)
    k_spline_cols(const __grid_constant__ InlinePlan inl, const void* plan_dev, int item0) {
  __shared__ float s_c[kColWarps][32], s_a[kColWarps][32];  // each warp's recursion ends
  const PlanView P = make_view(inl, plan_dev);
  const int item = item0 + (int)blockIdx.x;
  if (item >= P.h->ncolsegs) return;
  const SetDesc& S = P.sets[find_by(P.sets, P.h->nsets, item, 1)];
  const int W = S.W, H = S.H;
  const int ncb = (W + kColOut - 1) / kColOut, nrb = (H + kColRows - 1) / kColRows;
  const int local = item - S.colseg0;
  const int k = local / (ncb * nrb);
  const int rem = local - k * (ncb * nrb);
  const int rbk = rem / ncb, cb = rem - rbk * ncb;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const FrameDesc& F = P.frames[S.frame0 + k];
  // lane l solves source column cx = kColOut cb + ox + l (mirror-extended:
  // the coefficients of a mirrored column are the mirrored coefficients);
  // output column x = kColOut cb + l takes its taps from lanes l .. l + 3
  const int x = kColOut * cb + lane;
  int cx = x + F.ox;
  if ((unsigned)cx >= (unsigned)W) {
    const int p = 2 * W - 2;
    cx = cx < 0 ? -cx : cx;
    cx %= p;
    if (cx >= W) cx = p - cx;
  }
  const float* in = F.crow + cx;
  const int64_t ip = S.crow_pitch;
  const int y0 = rbk * kColRows + warp * 32;
  // rows outside [0, H) read the mirror-extended column (period 2H - 2)
  auto mirror = [&](int y) {
    int a = y < 0 ? -y : y;
    if (a >= H) {
      const int p = 2 * H - 2;
      a %= p;
      if (a >= H) a = p - a;
    }
    return a;
  };
  // the warp's 32 rows and, for the CTA's first / last warp, the 16 warm-up
  // rows above / below, all requested before the first is used
  const bool edge_warp = warp == 0 || warp == kColWarps - 1;
  const int yw = warp == 0 ? y0 - kColWarm : y0 + 32;
  float v[32], w[kColWarm];
  const int ylo = y0 - (warp == 0 ? kColWarm : 0),
            yhi = y0 + 32 + (warp == kColWarps - 1 ? kColWarm : 0);
  if (ylo >= 0 && yhi <= H) {
    const float* p = in + (int64_t)y0 * ip;
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __ldg(p + (int64_t)j * ip);
    if (edge_warp) {
      const float* q = in + (int64_t)yw * ip;
#pragma unroll
      for (int j = 0; j < kColWarm; ++j) w[j] = __ldg(q + (int64_t)j * ip);
    }
  } else {
    int iv[32], iw[kColWarm];
#pragma unroll
    for (int j = 0; j < 32; ++j) iv[j] = mirror(y0 + j);
#pragma unroll
    for (int j = 0; j < kColWarm; ++j) iw[j] = mirror(yw + j);
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __ldg(in + (int64_t)iv[j] * ip);
    if (edge_warp) {
#pragma unroll
      for (int j = 0; j < kColWarm; ++j) w[j] = __ldg(in + (int64_t)iw[j] * ip);
    }
  }
  // local recursions from zero: the causal end feeds the warp below, the
  // anti-causal start feeds the warp above (anything older is damped by z1^32)
  float yl[32];
  {
    float a = 0.0f;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      a = __fmaf_rn(kZ1, a, v[j]);
      yl[j] = a;
    }
    s_c[warp][lane] = a;
    float b = 0.0f;
#pragma unroll
    for (int j = 31; j >= 0; --j) b = __fmaf_rn(kZ1, b, v[j]);
    s_a[warp][lane] = b;
  }
  // at the CTA's top and bottom the carries come from warm-up rows
  float cin = 0.0f, ain = 0.0f;
  if (warp == 0) {
#pragma unroll
    for (int j = 0; j < kColWarm; ++j) cin = __fmaf_rn(kZ1, cin, w[j]);
  }
  if (warp == kColWarps - 1) {
#pragma unroll
    for (int j = kColWarm - 1; j >= 0; --j) ain = __fmaf_rn(kZ1, ain, w[j]);
  }
  __syncthreads();
  if (warp > 0) cin = s_c[warp - 1][lane];
  if (warp < kColWarps - 1) ain = s_a[warp + 1][lane];
  if (y0 >= H) return;  // (after the last shuffle partner has its data: none below)
  constexpr ZPow<32> zp{};
  // coefficients, then the horizontal taps from lanes l .. l + 3:
  // h(x, y) = sum_i wx_i c(x + ox + i, y), in the order the 4x4 evaluation uses
  const float wx0 = F.wx[0], wx1 = F.wx[1], wx2 = F.wx[2], wx3 = F.wx[3];
  const bool store = lane < kColOut && x < W;
  const int hpi = (int)S.coef_pitch;
  float* const out = F.coef + x;  // filtered frame (x, y) at (y + 2) * pitch + x
  float* const o = out + (int64_t)(y0 + 2) * hpi;
  const int ny = min(32, H - y0);
  float acc = ain;
#pragma unroll
  for (int j = 31; j >= 0; --j) {
    acc = __fmaf_rn(kZ1, acc, v[j]);
    const float yp = __fmaf_rn(zp.p[j + 1], cin, yl[j]);
    const float c = __fmul_rn(kSqrt3, __fsub_rn(__fadd_rn(yp, acc), v[j]));
    const float c1 = __shfl_down_sync(0xffffffffu, c, 1);
    const float c2 = __shfl_down_sync(0xffffffffu, c, 2);
    const float c3 = __shfl_down_sync(0xffffffffu, c, 3);
    float hh = wx0 * c;
    hh = __fmaf_rn(wx1, c1, hh);
    hh = __fmaf_rn(wx2, c2, hh);
    hh = __fmaf_rn(wx3, c3, hh);
    yl[j] = hh;
    if (store && j < ny) o[j * hpi] = hh;
  }
  // the 2-row mirrored border: h[-1] = h[1], h[-2] = h[2], h[H] = h[H-2],
  // h[H+1] = h[H-3] (the horizontal taps commute with the row mirror)
  if (store && (y0 < 3 || y0 + ny > H - 3)) {
    const int rows[4] = {1, 2, H - 2, H - 3}, mrow[4] = {-1, -2, H, H + 1};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int j = rows[r] - y0;
      if (j < 0 || j >= ny) continue;
      out[(int64_t)(mrow[r] + 2) * hpi] = select_at(yl, j);
    }
  }
}

cudaError_t launch_spline_rows(int e, const InlinePlan* inl, const void* plan_dev, int item0,
                               int count, cudaStream_t s, int stride) {  // (row block, frame group) items
  static bool opted[2] = {false, false};
  const size_t smem = rows_smem_bytes(e);
  cudaError_t err = cudaSuccess;
  if (e == 32) {
    if (!opted[0]) {
      err = cudaFuncSetAttribute(k_spline_rows<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
      if (err != cudaSuccess) return err;
      opted[0] = true;
    }
    k_spline_rows<32><<<count, 256, smem, s>>>(*inl, plan_dev, item0, stride);
  } else {
    if (!opted[1]) {
      err = cudaFuncSetAttribute(k_spline_rows<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
      if (err != cudaSuccess) return err;
      opted[1] = true;
    }
    k_spline_rows<64><<<count, 256, smem, s>>>(*inl, plan_dev, item0, stride);
  }
  return cudaGetLastError();
}

// One thread per 128-byte line of dead data: discard.global.L2 invalidates
// the line in L2 without writing it back (the data is never read again).
// Range i covers lines [first, first + lines) of the 128-byte-aligned base
// p + i * stride.
__global__ void k_discard_l2(const char* p, size_t first, size_t lines, int count,
                             size_t stride) {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  const size_t total = lines * (size_t)count;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t r = t / lines, l = t - r * lines;
    const char* a = p + r * stride + (first + l) * 128;
    asm volatile("discard.global.L2 [%0], 128;\n" ::"l"(a) : "memory");
  }
}

cudaError_t launch_discard_l2(const void* p, size_t bytes, int count, size_t stride,
                              cudaStream_t s) {
  if (count <= 0 || bytes == 0) return cudaSuccess;
  // lines wholly inside [p, p + bytes); stride is a multiple of 128 (or unused)
  const uintptr_t a = (uintptr_t)p, b = a + bytes;
  const uintptr_t first = (a + 127) / 128, last = b / 128;
  if (last <= first) return cudaSuccess;
  const uintptr_t base = (a / 128) * 128;
  const size_t lines = last - first;
  const size_t total = lines * (size_t)count;
  const int grid = (int)std::min<size_t>((total + 255) / 256, 4096);
  k_discard_l2<<<grid, 256, 0, s>>>((const char*)base, first - a / 128, lines, count, stride);
  return cudaGetLastError();
}

cudaError_t launch_spline_cols(const InlinePlan* inl, const void* plan_dev, int item0, int count,
                               cudaStream_t s) {  // (frame, 29 columns, kColRows rows) items
  k_spline_cols<<<count, kColRows, 0, s>>>(*inl, plan_dev, item0);
  return cudaGetLastError();
}

}  // namespace irp

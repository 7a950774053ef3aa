// common.cuh -- descriptors and device helpers shared by the sm_103a kernels.
//
// The fused path reduces frame sets tile by tile: one CTA owns one tile of
// the output grid of one set, walks the set's frames, calibrates and
// resamples each frame's source window into shared memory, and finally
// combines the per-pixel samples (sigma-clipped mean, median).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "irp.h"

namespace irp {

constexpr int kThreads = 256;  // 8 warps per CTA of the fused kernel

constexpr int kMaxInlineSets = 4;
constexpr int kMaxInlineFrames = 64;

// ST_BSPLINE: 4x4 cubic B-spline on padded coefficient frames; ST_BSPLINE_V:
// its vertical 4 taps on frames whose rows already carry the horizontal taps;
// ST_BSPLINE_T: column recursion and all 16 taps in the tile kernel, from the
// row-pass coefficients (k_spline_tile.cu).
// ST_CUBIC: Keys' cubic convolution, 4x4 taps on the calibrated raw frame.
enum Stencil : int {
  ST_NEAREST = 0, ST_BILINEAR = 1, ST_BSPLINE = 2, ST_BSPLINE_V = 3, ST_BSPLINE_T = 4,
  ST_CUBIC = 5
};
enum Source : int { SRC_RAW = 0, SRC_F32 = 1, SRC_F16 = 2 };

// Cubic-spline prefilter (Sec. 3.2.1's per-line tridiagonal system, solved in
// the parallel recursive form): c = sqrt(3) (y+ + y- - v), y+ and y- the causal
// and anti-causal first-order recursions with pole z1 = sqrt(3) - 2.
constexpr float kZ1 = -0.26794919243112270f;
constexpr float kSqrt3 = 1.7320508075688772f;
constexpr int kPrefHalo = 16;  // recursion warm-up; |z1|^17 / (1 - |z1|) < 3e-10
constexpr int kPrefTile = 64;  // prefilter output tile (square)

// Per-frame normalisation before the combine (workspace, 16 bytes): the FP64
// sum of the calibrated frame, and the factors every sample of the frame gets,
// x' = fma(x, na, nz): (1, m_0 - m_k) for a zero offset, (m_0 / m_k, 0) for a
// scale, m_k the frame's mean calibrated value and m_0 that of the set's
// first frame.
struct FrameNorm {
  double sum;
  float na, nz;
};

// One frame of a set, as the kernels see it (128 bytes).
struct FrameDesc {
  const void* src;     // raw uint16 frame (fused path) or FP32/F16 frame
  float* coef;         // FP32 spline coefficients of the frame (workspace) or null
  int32_t ox, oy;      // integer tap origin: the stencil's first tap is at
                       // (x + ox, y + oy) for output pixel (x, y)
  float fx, fy;        // fractional offsets in [0, 1)
  float t;             // exposure time (s)
  float scale, offset; // F16 frames: value = h * scale + offset
  int32_t vx0, vx1;    // sample valid iff vx0 <= x <= vx1 ...
  int32_t vy0, vy1;    //              ... and vy0 <= y <= vy1
  float wx[4], wy[4];  // stencil weights (bilinear: 1-f, f; spline: beta3)
  int32_t flags;       // bit 0: raw frame 16-byte aligned with a pitch of 8k elements;
                       // bit 1: 8-byte aligned with a pitch of 4k elements
  float* crow;         // row-pass spline coefficients (workspace) or null
  const uint32_t* bad; // bad-pixel bits of the frame (masked spline sets, workspace) or null
  int32_t last_tap;    // bit 0 (1): the last tap along x (y) has non-zero weight, fx > 0
                       // (fy > 0) in FP64; the FP32 weights may round such a weight to 0
  int32_t pad1;
  struct FrameNorm* norm;  // per-frame normalisation record (workspace) or null
};
static_assert(sizeof(FrameDesc) == 128, "FrameDesc layout");

// One frame set (224 bytes).
struct SetDesc {
  int32_t W, H, n, frame0;       // frame0: index of frame 0 in the frame table
  int64_t src_pitch;             // elements of the frames' element type
  const float* bias;
  const float* dark;
  const float* flat;
  int64_t master_pitch;
  const double* flat_sum;        // FP64 sum of the flat (normalise) or null
  float* mean_out;
  float* median_out;
  uint16_t* nkept_out;
  float* stack_out;
  int64_t out_pitch;
  int32_t tiles_x, tiles_y;      // output tiles (tile_cols x tile_rows)
  int32_t tile0;                 // first work item of this set
  int32_t mwin_w, mwin_h;        // master union window (0 = per-frame masters)
  int32_t mox, moy;              // union window origin relative to the tile
  int32_t ptiles_x, ptiles_y;    // prefilter tiles (kPrefTile squared)
  int32_t ptile0;                // first prefilter work item of this set
  const uint32_t* ready_flag;
  uint32_t ready_value;
  int32_t pframes;               // frames per prefilter work item
  int64_t coef_pitch;            // padded spline-coefficient frames: (H+4) rows
  int64_t crow_pitch;            // row-pass coefficient frames (spath 1)
  int32_t row0;                  // first row-pass work item (row block x frame chunk)
  int32_t colseg0;               // first column-pass work item
  int32_t mflags;                // bit 0: masters 16-byte aligned, pitch of 4k elements;
                                 // bit 1: premerged master window (one exposure time, no mask)
  int32_t spath;                 // spline prefilter: 0 tiled, 1 row + column passes
  const uint8_t* mask;           // bad-pixel mask master or null
  int64_t mask_pitch;
  float saturation;              // raw level marking a pixel bad (+inf: none)
  int32_t masked;                // 1: mask or saturation level in use
  int32_t stack_only;            // 1: write stack_out only (a chunk of a deeper set)
  int32_t rgroup;                // frames per row-pass work item (at most kRowGroup)
  int64_t bad_pitch;             // words per row of the bad-pixel bits (masked spline sets)
  const FrameNorm* norm_ref;     // normalisation record of the set's first frame, or null
};
static_assert(sizeof(SetDesc) == 240, "SetDesc layout");

struct PlanHeader {
  int32_t nsets, nframes, nitems, stencil;
  int32_t max_n, persistent, spin_limit, src;
  float kappa_lo, kappa_hi;
  int32_t max_iter, center, ddof;
  int32_t smem_samples;          // floats reserved per CTA for samples
  int32_t smem_master;           // float4 entries reserved per CTA for master windows
  int32_t npitems;               // tiled prefilter work items (spline)
  int32_t nrows, ncolsegs;       // row-pass and column-pass work items (spline)
  int32_t frame_norm;            // per-frame normalisation: 0 none, 1 zero, 2 scale
  int32_t pad;
  uint32_t* status;              // device status word (workspace)
  uint32_t* counter;             // persistent work counter (workspace)
};
static_assert(sizeof(PlanHeader) % 16 == 0 && sizeof(PlanHeader) <= 128, "PlanHeader layout");

// Plan passed by value as a kernel parameter for small launches.
struct InlinePlan {
  PlanHeader h;
  SetDesc sets[kMaxInlineSets];
  FrameDesc frames[kMaxInlineFrames];
};

// Plan in global memory (workspace) for large launches: PlanHeader (128 B),
// then SetDesc[nsets], then FrameDesc[nframes].
struct PlanView {
  const PlanHeader* h;
  const SetDesc* sets;
  const FrameDesc* frames;
};

__host__ __device__ inline size_t plan_sets_offset() { return 128; }
__host__ __device__ inline size_t plan_frames_offset(int nsets) {
  return 128 + (size_t)nsets * sizeof(SetDesc);
}
__host__ __device__ inline size_t plan_total_bytes(int nsets, int nframes) {
  return plan_frames_offset(nsets) + (size_t)nframes * sizeof(FrameDesc);
}

// Workspace header (first 256 bytes of every workspace).
struct WsHeader {
  uint32_t status;
  uint32_t counters[31];  // persistent work counters, one per sub-plan
  uint8_t pad[128];
};
static_assert(sizeof(WsHeader) == 256, "WsHeader layout");

__device__ __forceinline__ void latch_status(uint32_t* status, uint32_t code) {
  if (status) atomicCAS(status, 0u, code);
}

// Whole-sample symmetric index into [0, N).
__device__ __forceinline__ int mirror_index(int i, int N) {
  if (N <= 1) return 0;
  if (i >= 0 && i < N) return i;
  int period = 2 * (N - 1);
  int r = i % period;
  if (r < 0) r += period;
  return r >= N ? period - r : r;
}

__device__ __forceinline__ float bspline3(float t) {
  float a = fabsf(t);
  if (a < 1.0f) return 2.0f / 3.0f - a * a + 0.5f * a * a * a;
  if (a < 2.0f) {
    float b = 2.0f - a;
    return b * b * b * (1.0f / 6.0f);
  }
  return 0.0f;
}

// Locates the set owning work item ``item`` (sets ordered by tile0).
__device__ __forceinline__ int find_set(const SetDesc* sets, int nsets, int item) {
  int lo = 0, hi = nsets - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (sets[mid].tile0 <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Bounded wait for a set's ready flag; returns false (and latches
// IRP_ERR_TIMEOUT) if the flag did not reach the value in ``limit`` polls.
__device__ __forceinline__ bool wait_ready(const uint32_t* flag, uint32_t value, int limit,
                                           uint32_t* status) {
  if (!flag) return true;
  for (int i = 0; i < limit; ++i) {
    uint32_t v = *((volatile const uint32_t*)flag);
    if ((int32_t)(v - value) >= 0) return true;
    __nanosleep(1000);
  }
  latch_status(status, IRP_ERR_TIMEOUT);
  return false;
}

// ---------------------------------------------------------------------------
// Host-side launchers and geometry (implemented in the kernel files).
// ---------------------------------------------------------------------------
int reduce_bucket(int n);                  // register bucket (sort size) for n frames
int rows_per_warp(int bucket, int stencil, int requested);  // requested if valid, else default
int tile_cols(int stencil);                // output columns per tile
int tile_rows(int bucket, int py);         // output rows per tile
size_t reduce_smem_bytes(int src, int stencil, int py, int max_n, int mwin_f4);
int reduce_occupancy(int bucket, int py, int stencil, size_t smem);
cudaError_t launch_reduce(int bucket, int py, int stencil, const InlinePlan* inl,
                          const void* plan_dev, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_prefilter_raw(const InlinePlan* inl, const void* plan_dev, int grid,
                                 cudaStream_t s);

}  // namespace irp

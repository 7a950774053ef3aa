// unfused.h -- argument blocks and launchers of the separate-step kernels.
#pragma once

#include "combine.cuh"
#include "common.cuh"

namespace irp {

constexpr int kCalibChunk = 256;   // frames per calibration launch (times by value)
constexpr int kShiftChunk = 64;    // frames per shift launch (descriptors by value)
constexpr float kF16Range = 16384.0f;  // |h| bound of FP16 stacks (4x headroom)

// Rows per stats block: about 16K pixels per block.
__host__ __device__ inline int stats_rows(int W, int H) {
  int r = 16384 / (W > 0 ? W : 1);
  r = r < 1 ? 1 : r;
  return r > H ? H : r;
}

struct FrameStats {  // 32 bytes per frame, workspace
  double sum, sumsq;
  long long count;
  int min_key, max_key;
};

struct CalibArgs {
  const uint16_t* raw;
  int64_t raw_pitch, raw_frame_stride;
  int W, H, k0;
  int vec;                  // raw, masters (and outputs): 4-pixel vector loads and stores
  const float* bias;
  const float* dark;
  const float* flat;
  int64_t master_pitch;
  const double* flat_sum;   // null: no flat normalisation
  uint32_t* status;
  float t[kCalibChunk];
};

struct ShiftArgs {
  const void* in;
  int64_t in_pitch, in_fstride;
  int W, H, k0, pad;
  void* out;
  int64_t out_pitch, out_fstride;
  uint8_t* valid_out;
  int64_t coef_pitch;   // padded spline-coefficient frames ((H+4) rows)
  FrameDesc frames[kShiftChunk];
};

struct CombineArgs {
  const void* stack;         // null: samples from horizontally filtered spline rows
  const FrameDesc* frames;   // ... of these frames (device), when stack is null
  int64_t coef_pitch;        // ... with this row pitch
  int64_t pitch, fstride;
  int W, H, n, frame_norm;   // frame_norm: apply the frames' normalisation (filtered rows)
  const float* scale;
  const float* offset;
  const uint8_t* valid;
  ClipArgs clip;
  float* mean_out;
  float* median_out;
  uint16_t* nkept_out;
  uint8_t* reject_out;
  int64_t out_pitch;
};

cudaError_t launch_stats_init(FrameStats* st, int n, cudaStream_t s);
cudaError_t launch_stats_raw(const CalibArgs& a, int nk, FrameStats* st, cudaStream_t s);
// Eight-pixel forms (rows of raw, masters and outputs on 8-pixel boundaries):
// the FP16 scaling sums (sum, minimum, maximum) and calibration, each block
// over every frame of the launch.
cudaError_t launch_f16_stats8(const CalibArgs& a, int nk, FrameStats* st, cudaStream_t s);
cudaError_t launch_calibrate8(const CalibArgs& a, int nk, bool f16, void* out, int64_t out_pitch,
                              int64_t out_fstride, const float* scale, const float* offset,
                              cudaStream_t s);
// Sums into FrameStats (st != null) or into the separate arrays sum/sumsq/count.
cudaError_t launch_stats_frames(const void* frames, int64_t pitch, int64_t fstride, int W, int H,
                                int n, bool f16, const float* scale, const float* offset,
                                double* sum, double* sumsq, long long* count, FrameStats* st,
                                cudaStream_t s);
cudaError_t launch_f16_scaling(const FrameStats* st, int n, float* scale, float* offset,
                               cudaStream_t s);
// Per-frame normalisation of a (sub-)plan: the FP64 sums of its calibrated raw
// frames into their FrameNorm records (zeroed by the caller), then the factors.
cudaError_t launch_frame_norm(const InlinePlan* inl, const void* plan_dev, int nframes,
                              int max_row_blocks, cudaStream_t s);
cudaError_t launch_calibrate(const CalibArgs& a, int nk, bool f16, void* out, int64_t out_pitch,
                             int64_t out_fstride, const float* scale, const float* offset,
                             cudaStream_t s);
// vec: outputs (and validity bytes) 16-byte (FP32) or 8-byte (FP16) aligned
// with pitches of 4k pixels, so that four outputs leave as one store
cudaError_t launch_shift(const ShiftArgs& a, int nk, int stencil, bool f16, int vec,
                         cudaStream_t s);
cudaError_t launch_prefilter_frames(const InlinePlan* inl, int grid, bool f16, cudaStream_t s);
cudaError_t launch_combine(const CombineArgs& a, bool f16, cudaStream_t s);
// More than IRP_MAX_FRAMES frames (up to IRP_MAX_WIDE_FRAMES): a group of lanes per pixel.
cudaError_t launch_combine_wide(const CombineArgs& a, bool f16, cudaStream_t s);

}  // namespace irp

/*
 * irp.h -- C ABI of the GB300 image-reduction library.
 *
 * The library implements the data-parallel part of the image reduction of
 * Niwano et al., "GPU-accelerated Image Reduction Pipeline" (PASJ 2020):
 *
 *   Sec. 2.1 / 2.2  bias subtraction, dark subtraction and flat fielding of raw
 *                   16-bit CCD frames (the integers become floating point at the
 *                   bias subtraction);
 *   Sec. 2.1 / 2.2  alignment of the dithered frames by sub-pixel shifting with
 *                   bicubic-spline interpolation (also nearest and bilinear,
 *                   named as cheaper alternatives in Sec. 3.2.1);
 *   Sec. 2.1 / 2.2  co-adding by a sigma-clipped mean, plus the median.
 *
 * Conventions shared by every entry point
 *   - Images are row-major, x (column) fastest.  Pitches and frame strides are
 *     in ELEMENTS of the buffer's own type.
 *   - Every device buffer is allocated and owned by the caller.  Host arrays
 *     (offsets, exposure times, frame pointer tables) are read during the call
 *     only.  No entry point allocates device memory; irp_reduce_set builds its
 *     launch plan in a temporary host buffer, irp_plan_encode in the caller's.
 *   - Offsets: output pixel (x, y) samples frame k at (x + dx[k], y + dy[k]).
 *     The offset is split as dx = ix + fx, ix = floor(dx), fx in [0, 1).
 *   - A sample is valid iff every tap with non-zero weight lies inside the
 *     frame (nearest, bilinear, cubic convolution) or the source position lies inside
 *     [0, W-1] x [0, H-1] (cubic spline).  Invalid samples do not enter the
 *     combination; a pixel with no valid sample gets NaN (mean, median).
 *   - The cubic spline is the interpolating cubic B-spline with mirror
 *     (whole-sample symmetric) boundary conditions (Sec. 3.1.1, Sec. 3.2.1).
 *   - Calibration: v = (raw - bias - dark_rate * t) * (flat_norm / flat) in
 *     FP32, flat_norm = 1 or the FP64 mean of the flat (normalize_flat).
 *   - Sigma clip: up to max_iter passes; centre = mean (or median) of the
 *     survivors, sigma^2 = sum (x - centre)^2 / (m - ddof); x is rejected if
 *     centre - x > kappa_lo sigma or x - centre > kappa_hi sigma; rejection is
 *     cumulative; the loop stops when nothing is rejected or sigma = 0.  The
 *     output is the mean of the survivors.  The median is taken over all valid
 *     samples before clipping (even count: mean of the two middle values).
 *   - stream is a cudaStream_t (NULL = legacy default stream).  Work is
 *     enqueued asynchronously; arguments are validated before anything is
 *     enqueued, and a non-OK status means nothing was enqueued.
 *   - Errors detected on the device (a non-finite or non-positive flat value,
 *     a bounded wait that ran out) are latched into the status word at the
 *     start of the caller's workspace and reported by irp_sync_status().
 *   - Workspaces: device memory, 256-byte aligned, owned by the caller.  The
 *     first 256 bytes (status word, work counters) must be zero before the
 *     workspace is first used; the library keeps them consistent afterwards
 *     (irp_sync_status clears a latched status).  Calls that share a
 *     workspace must be ordered (same stream or synchronised).
 */
#ifndef IRP_H
#define IRP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IRP_VERSION 10000      /* 1.0.0 */
#define IRP_MAX_FRAMES 64      /* frames per set on the per-thread register combine */
#define IRP_MAX_WIDE_FRAMES 1024 /* frames per set; from IRP_MAX_FRAMES + 1 on, a
                                    group of lanes combines each pixel (the paper's
                                    bands hold 180 frames, Sec. 3.2.1) */

typedef enum {
  IRP_OK = 0,
  IRP_ERR_INVALID_ARG = 1,   /* null required pointer, bad size, bad enum */
  IRP_ERR_ALIGNMENT = 2,     /* a buffer is not aligned to its element size */
  IRP_ERR_WORKSPACE = 3,     /* workspace missing or smaller than required */
  IRP_ERR_UNSUPPORTED = 4,   /* a valid request the library does not implement */
  IRP_ERR_BAD_MASTER = 5,    /* device: flat value <= 0 or not finite */
  IRP_ERR_CUDA = 6,          /* a CUDA runtime call failed */
  IRP_ERR_TIMEOUT = 7,       /* device: a bounded wait gave up */
  IRP_ERR_BAD_STATISTIC = 8  /* device: a frame's mean level is 0 or not finite (scale
                                normalisation) */
} irp_status;

/* IRP_INTERP_CUBIC: Keys' cubic convolution (a = -1/2), 4 x 4 taps on the
 * calibrated data with no prefilter; a cheaper alternative to the cubic
 * spline (Keys, IEEE Trans. ASSP 29, 1981).  Its samples are valid when every
 * tap with non-zero weight lies inside the frame, as for bilinear. */
typedef enum {
  IRP_INTERP_NEAREST = 0, IRP_INTERP_BILINEAR = 1, IRP_INTERP_SPLINE3 = 2, IRP_INTERP_CUBIC = 3
} irp_interp;

/* Element type of an intermediate (calibrated or aligned) stack.
 * IRP_F16_SCALED: value = (float)h * scale[k] + offset[k], h an IEEE half. */
typedef enum { IRP_F32 = 0, IRP_F16_SCALED = 1 } irp_stack_dtype;

typedef struct {
  float kappa_lo, kappa_hi;  /* rejection thresholds in sigma (3, 3)        */
  int max_iter;              /* rejection passes (3)                        */
  int center;                /* 0: mean, 1: median                          */
  int ddof;                  /* 0: population sigma                         */
} irp_clip_params;

/* ---------------------------------------------------------------------------
 * irp_calibrate -- Sec. 2.1 bias subtraction, dark subtraction, flat fielding.
 *   raw      [n][H][raw_pitch] uint16 frames, frame k at raw + k*raw_frame_stride
 *   bias, dark_rate, flat  [H][master_pitch] FP32 masters (dark in ADU/s)
 *   exptime_host  [n] exposure times in s (host memory)
 *   out      dt == IRP_F32:        float [n][H][out_pitch], frame stride out_frame_stride
 *            dt == IRP_F16_SCALED: half  [n][H][out_pitch]; scale_out/offset_out
 *            [n] (device) receive the per-frame scaling chosen on the device:
 *            offset = FP64 mean of the frame, scale = power of two with
 *            max |v - offset| / scale <= 16384.
 *   workspace  >= irp_calibrate_workspace_size(n) bytes, 256-byte aligned.
 * ------------------------------------------------------------------------- */
irp_status irp_calibrate(const uint16_t* raw, int64_t raw_pitch, int64_t raw_frame_stride,
                         int W, int H, int n,
                         const float* bias, const float* dark_rate, const float* flat,
                         int64_t master_pitch, const float* exptime_host, int normalize_flat,
                         void* out, int64_t out_pitch, int64_t out_frame_stride,
                         irp_stack_dtype dt, float* scale_out, float* offset_out,
                         void* workspace, size_t ws_bytes, void* stream);
size_t irp_calibrate_workspace_size(int n);

/* ---------------------------------------------------------------------------
 * irp_frame_stats -- FP64 frame-wide sums (sky level, normalisation).
 *   frames   F32 or F16_SCALED [n][H][pitch]; NaN entries are skipped.
 *   sum_out, sumsq_out [n] (device, double), count_out [n] (device, int64).
 * ------------------------------------------------------------------------- */
irp_status irp_frame_stats(const void* frames, int64_t pitch, int64_t frame_stride,
                           int W, int H, int n, irp_stack_dtype dt,
                           const float* scale, const float* offset,
                           double* sum_out, double* sumsq_out, int64_t* count_out,
                           void* stream);

/* ---------------------------------------------------------------------------
 * irp_shift -- Sec. 2.1 alignment: resamples each calibrated frame onto the
 * reference grid.  in/out have the same dtype; F16_SCALED frames keep their
 * per-frame scale/offset (interpolation weights sum to one).  Invalid samples
 * are written as NaN; valid_out [n][H][out_pitch] (nullable) receives 0/1.
 *   dx_host, dy_host [n] offsets in pixels (host).
 *   workspace >= irp_shift_workspace_size(W, H, n, interp) bytes (the spline
 *   coefficients, n*W*H floats, for IRP_INTERP_SPLINE3).
 * ------------------------------------------------------------------------- */
irp_status irp_shift(const void* in, int64_t in_pitch, int64_t in_frame_stride,
                     int W, int H, int n, irp_stack_dtype dt,
                     const float* scale, const float* offset,
                     const double* dx_host, const double* dy_host, irp_interp interp,
                     void* out, int64_t out_pitch, int64_t out_frame_stride,
                     uint8_t* valid_out, void* workspace, size_t ws_bytes, void* stream);
size_t irp_shift_workspace_size(int W, int H, int n, irp_interp interp);

/* ---------------------------------------------------------------------------
 * irp_combine -- Sec. 2.1 co-adding: sigma-clipped mean and median of an
 * aligned stack [n][H][pitch] (F32 or F16_SCALED; NaN = invalid sample).
 *   valid    nullable [n][H][pitch] uint8 mask, 0 excludes the sample.
 *   mean_out, median_out  [H][out_pitch] float (either may be NULL).
 *   nkept_out  nullable [H][out_pitch] uint16 survivors of the clip.
 *   reject_out nullable [n][H][out_pitch] uint8, 1 where a valid sample was
 *              rejected by the clip (debug output).
 *   n <= IRP_MAX_WIDE_FRAMES: up to IRP_MAX_FRAMES one thread sorts a pixel's
 *   samples in registers; deeper stacks take 4 to 32 lanes per pixel
 *   (bitonic sort over the lanes, the same clip), with identical semantics.
 * ------------------------------------------------------------------------- */
irp_status irp_combine(const void* stack, int64_t pitch, int64_t frame_stride,
                       int W, int H, int n, irp_stack_dtype dt,
                       const float* scale, const float* offset, const uint8_t* valid,
                       const irp_clip_params* clip,
                       float* mean_out, float* median_out, uint16_t* nkept_out,
                       uint8_t* reject_out, int64_t out_pitch, void* stream);

/* ---------------------------------------------------------------------------
 * irp_reduce_set -- the fused path: calibration, alignment and combination of
 * one or more frame sets, each raw pixel read from HBM once (bilinear and
 * nearest; cubic spline computes the spline coefficients of every calibrated
 * frame into the workspace first and then resamples and combines them).
 * A cubic-spline set whose frames take the row pass (W from 34 to 8192, H at
 * least 34) is reduced from the row-pass coefficients by one tile kernel,
 * which keeps each tile's samples on chip: up to IRP_MAX_FRAMES frames, and
 * masked sets up to 256 frames (a group of 4 or 8 lanes then combines a
 * pixel).  Any other set of more than IRP_MAX_FRAMES frames (up to
 * IRP_MAX_WIDE_FRAMES) is resampled in chunks of at most 16 frames into its
 * aligned FP32 stack [n][H][pitch] -- stack_out when given (pitch
 * out_pitch), else the workspace (pitch W rounded up to 32) -- and the stack
 * is then combined by a group of lanes per pixel; an unmasked cubic-spline
 * set on the row and column passes writes no stack unless stack_out is
 * given: its combine forms each sample from the horizontally filtered rows.
 * irp_workspace_size accounts for what each set needs.
 * ------------------------------------------------------------------------- */
typedef struct {
  const uint16_t* const* frames;  /* host array of n device pointers           */
  int64_t raw_pitch;              /* elements, shared by the set's frames       */
  int W, H, n;
  const double* dx;               /* host [n] */
  const double* dy;               /* host [n] */
  const float* exptime;           /* host [n], seconds */
  const float* bias;              /* device [H][master_pitch] */
  const float* dark_rate;         /* device, ADU/s */
  const float* flat;              /* device */
  int64_t master_pitch;
  float* mean_out;                /* device [H][out_pitch], may be NULL */
  float* median_out;              /* device [H][out_pitch], may be NULL */
  uint16_t* nkept_out;            /* device, nullable */
  int64_t out_pitch;
  float* stack_out;               /* device [n][H][out_pitch] aligned samples, NaN
                                     = invalid; nullable (debug) */
  const uint32_t* ready_flag;     /* device, nullable: the set's tiles wait until
                                     *ready_flag >= ready_value (bounded wait) */
  uint32_t ready_value;
  /* Bad-pixel masking (Sec. 2.1, bad-pixel masking before alignment): a source
   * pixel is bad when mask[y*mask_pitch + x] != 0 or its raw value is at least
   * `saturation`; a sample whose taps with non-zero weight include a bad pixel
   * is invalid (left out of the combine, NaN in stack_out).  Every
   * resampler; with the cubic spline only for sets on the row pass (W from
   * 34 to 8192, H at least 34) of at most 256 frames, others returning
   * IRP_ERR_UNSUPPORTED. */
  const uint8_t* mask;            /* device [H][mask_pitch] uint8, nullable */
  int64_t mask_pitch;             /* elements (>= W when mask is set) */
  float saturation;               /* raw ADU; 0 = no saturation test */
} irp_set;

typedef struct {
  irp_interp interp;
  irp_clip_params clip;
  int normalize_flat;             /* divide the flat by its FP64 mean */
  int persistent;                 /* 1: persistent CTAs pulling (set, tile) work
                                     items from an atomic counter, longest first */
  int max_ctas;                   /* persistent grid size; 0 = SMs x occupancy  */
  int wait_spin_limit;            /* bounded-wait polls before IRP_ERR_TIMEOUT; 0 = default */
  int rows_per_warp;              /* tile height / 8: 0 = default of the frame-count
                                     bucket and stencil (4 up to 16 frames; 2 up to
                                     40 frames, and above for the Keys stencil and
                                     the tiled spline; else 1), or the bucket's
                                     other value when it is the shorter and the
                                     default tiles of a group would give fewer than
                                     two CTAs per SM; the other accepted value is 2
                                     (resp. 1; resp. 2); anything else falls back
                                     to the default */
  int frame_norm;                 /* per-frame normalisation before the combine (a
                                     combine variant; the paper has none): 0 none;
                                     1 zero: each sample of frame k gets m_0 - m_k
                                     added; 2 scale: it is multiplied by m_0 / m_k;
                                     m_k = the FP64 mean of frame k's calibrated
                                     values over the whole frame, frame 0 the set's
                                     first.  The means take one more read of the raw
                                     frames.  With scale, a mean of 0 or not finite
                                     latches IRP_ERR_BAD_STATISTIC.  stack_out holds
                                     the normalised samples. */
  int spline_onchip;              /* cubic spline, unmasked sets on the row pass
                                     (34 <= W <= 8192, H >= 34, up to IRP_MAX_FRAMES
                                     frames): 0 = row pass, column pass (the
                                     filtered rows in the workspace) and the
                                     reduction of the vertical taps, the faster
                                     form; 1 = row pass, then one tile kernel that
                                     solves the columns and combines on chip, with
                                     the row-pass frames kept in L2: about 1.2x
                                     the algorithmic DRAM bytes instead of about
                                     4x, for callers that share HBM bandwidth.
                                     Masked sets always take the tile kernel. */
} irp_reduce_params;

size_t irp_workspace_size(const irp_set* sets, int nsets, const irp_reduce_params* p);
irp_status irp_reduce_set(const irp_set* sets, int nsets, const irp_reduce_params* p,
                          void* workspace, size_t ws_bytes, void* stream);

/* Two-step form of irp_reduce_set for CUDA-graph capture: irp_plan_encode
 * writes the launch plan (descriptors, work list) into a caller-owned host
 * buffer, pure host work; irp_plan_launch copies it into the workspace with
 * one cudaMemcpyAsync and launches.  With plan_host in pinned memory the
 * launch is capturable, and a captured graph re-reads plan_host at every
 * replay, so the caller may re-encode into it between replays. */
size_t irp_plan_bytes(const irp_set* sets, int nsets, const irp_reduce_params* p);
irp_status irp_plan_encode(const irp_set* sets, int nsets, const irp_reduce_params* p,
                           void* plan_host, size_t plan_bytes, void* workspace,
                           size_t ws_bytes);
irp_status irp_plan_launch(const void* plan_host, size_t plan_bytes, void* workspace,
                           size_t ws_bytes, void* stream);

/* irp_reduce_set_noalloc -- irp_reduce_set for callers that cannot allocate
 * device memory.  The paper has no counterpart; this is a deployment aid.
 *
 * Some callers cannot create a workspace: a real-time reduction loop that
 * reserves all device memory at start-up and must not allocate afterwards
 * (an allocation can stall for milliseconds or fail once memory is
 * fragmented), or a host framework that owns the device memory pool and hands
 * a plug-in only its input and output buffers.  This entry point takes the
 * same sets and parameters as irp_reduce_set but uses a scratch area of
 * IRP_NOALLOC_SCRATCH_BYTES that the library holds in a static device array;
 * every GPU that loads the library keeps that array until the process exits.
 * It allocates no device memory: it calls no cudaMalloc, cudaFree or other
 * allocating CUDA or library routine.
 *   - The caller still passes all inputs and outputs (irp_set).
 *   - status_out (device, nullable) receives the call's device status word
 *     (IRP_OK, IRP_ERR_BAD_MASTER, IRP_ERR_TIMEOUT) when the call's work
 *     completes on the stream.
 *   - Requests whose workspace (irp_workspace_size) exceeds
 *     IRP_NOALLOC_SCRATCH_BYTES, or whose plan exceeds the call's fixed host
 *     plan buffer, return IRP_ERR_WORKSPACE with nothing enqueued; use
 *     irp_reduce_set for those.
 *   - A plan of more than 4 sets or 64 frames in one frame-count group, or
 *     with a set deeper than IRP_MAX_FRAMES, is copied to the device from a
 *     buffer on the call's own stack.  While `stream` is being captured such
 *     a request returns IRP_ERR_UNSUPPORTED with nothing enqueued, since the
 *     recorded copy would read that buffer after the call has returned.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current.
 *   - All calls on a device share the one array, which keeps the contents of
 *     the last call; each call clears the status word and work counters
 *     before its kernels run.  Calls whose work overlaps on the GPU (other
 *     streams, other host threads without ordering) race on the array. */
#define IRP_NOALLOC_SCRATCH_BYTES ((size_t)8 << 20)
irp_status irp_reduce_set_noalloc(const irp_set* sets, int nsets, const irp_reduce_params* p,
                                  uint32_t* status_out, void* stream);

/* irp_reduce_set_host -- irp_reduce_set with the raw frames and the results
 * in host memory (Sec. 2.2: the frames are read into host memory and sent to
 * the GPU; the results come back to be written out).
 *   sets  as for irp_reduce_set: the device buffers that receive the frames
 *         (sets[i].frames) and the results (mean_out, median_out, nkept_out).
 *   io    [nsets] host side of each set:
 *           frames  host array of n host pointers, raw uint16 [H][pitch]
 *                   (page-locked memory lets the copies overlap the work);
 *           mean, median, nkept  host [H][out_pitch] destinations, each
 *                   nullable, and only with the matching device output set.
 *   workspace  >= irp_workspace_size(&sets[i], 1, p) for every i.
 * For each set in turn: its frames are copied to the device on an upload
 * stream, the set is reduced on `stream` once they have landed, and its
 * results are copied back on a download stream.  Set i+1 is uploaded while
 * set i is reduced, and set i's results return while set i+1 is reduced.
 * Both copy streams are the library's own (one pair per device, created on
 * first use); they fork from and join back into `stream` through events, so
 * the call is ordered on `stream` like any other, and the results are in
 * host memory once `stream` has reached the call's end.  No device memory
 * is allocated.  Validation errors return before anything is enqueued. */
typedef struct {
  const uint16_t* const* frames;  /* host array of n host pointers            */
  int64_t pitch;                  /* elements, shared by the set's frames     */
  float* mean;                    /* host, nullable */
  float* median;                  /* host, nullable */
  uint16_t* nkept;                /* host, nullable */
  int64_t out_pitch;              /* elements (>= W when an output is set)   */
} irp_host_io;

irp_status irp_reduce_set_host(const irp_set* sets, int nsets, const irp_host_io* io,
                               const irp_reduce_params* p, void* workspace, size_t ws_bytes,
                               void* stream);

/* Synchronises the stream, returns and clears the device status latched in
 * the workspace's status word. */
irp_status irp_sync_status(void* workspace, void* stream);

const char* irp_status_string(irp_status s);
/* Name and description of the CUDA error behind the last IRP_ERR_CUDA
 * returned on the calling thread ("" if none). */
const char* irp_last_cuda_error(void);
int irp_version(void);

/* Number of SMs of the current device (autotuning helper). */
int irp_device_sm_count(void);

/* Launch tracing: while enabled, every kernel the library launches is
 * bracketed by CUDA events recorded on its stream.  irp_profile_read
 * synchronises those events, writes per kernel kind the summed device time
 * (ms) and the launch count, clears the record and returns the number of
 * kinds written (at most max_kinds; kinds are the IRP_KERNEL_* values). */
enum {
  IRP_KERNEL_REDUCE = 0,     /* fused calibrate/resample/combine tile kernel */
  IRP_KERNEL_PREFILTER = 1,  /* spline coefficients of raw frames            */
  IRP_KERNEL_STATS = 2,      /* FP64 frame and master sums                   */
  IRP_KERNEL_CALIBRATE = 3,
  IRP_KERNEL_SHIFT = 4,      /* includes the spline prefilter of irp_shift   */
  IRP_KERNEL_COMBINE = 5,
  IRP_KERNEL_KINDS = 6
};
void irp_profile_enable(int on);
int irp_profile_read(double* ms_out, int64_t* launches_out, int max_kinds);

#ifdef __cplusplus
}
#endif
#endif /* IRP_H */

// api.cu -- the C ABI declared in include/irp.h.
//
// Host responsibilities: validate arguments before anything is enqueued,
// split every frame offset in FP64 into an integer tap origin, fractional
// weights and a validity range, build the launch plan (set and frame
// descriptors), and launch the kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "prefilter.cuh"
#include "spline.h"
#include "unfused.h"

using namespace irp;

namespace {

constexpr size_t kAlign = 256;
constexpr uint32_t kPlanMagic = 0x49525031u;  // "IRP1"
constexpr int kMaxSub = 24;  // one sub-plan per bucket (and spline path) at most
constexpr int kDefaultSpin = 1 << 20;  // polls of 1 us: about one second

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// ------------------------------------------------------------------ tracing
struct TraceRec {
  int kind;
  cudaEvent_t a, b;
};
struct Tracer {
  bool on = false;
  std::vector<TraceRec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};
Tracer& tracer() {
  static Tracer t;
  return t;
}

// Brackets the launches issued between construction and destruction.
struct TraceScope {
  int kind;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  TraceScope(int k, cudaStream_t st) : kind(k), s(st) {
    if (tracer().on) {
      a = tracer().get();
      cudaEventRecord(a, s);
    }
  }
  ~TraceScope() {
    if (a) {
      cudaEvent_t b = tracer().get();
      cudaEventRecord(b, s);
      tracer().recs.push_back(TraceRec{kind, a, b});
    }
  }
};
inline bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }
thread_local char g_last_cuda_error[256] = "";
inline irp_status note_cuda(cudaError_t e) {
  snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s: %s", cudaGetErrorName(e),
           cudaGetErrorString(e));
  return IRP_ERR_CUDA;
}
inline irp_status cuda_status(cudaError_t e) { return e == cudaSuccess ? IRP_OK : note_cuda(e); }

// Offset split along one axis: sample of output coordinate p is at
// (p + o) + tap, o the integer origin; valid iff v0 <= p <= v1.
struct Axis {
  int o;
  float f;
  int v0, v1;
  float w[4];
};

bool split_axis(double d, int N, int interp, Axis& a) {
  if (!std::isfinite(d) || std::fabs(d) > 1.0e9) return false;
  const double fl = std::floor(d);
  const double f = d - fl;  // exact in FP64
  const int ifl = (int)fl;
  a.f = (float)f;
  for (int i = 0; i < 4; ++i) a.w[i] = 0.0f;
  if (interp == IRP_INTERP_NEAREST) {
    // nearest integer to (p + ifl) + f, halves away from zero
    if (f < 0.5) {
      a.o = ifl;
      a.v0 = -ifl;
      a.v1 = N - 1 - ifl;
    } else if (f > 0.5) {
      a.o = ifl + 1;
      a.v0 = -ifl - 1;
      a.v1 = N - 2 - ifl;
    } else {  // p + ifl + 0.5 rounds up iff p + ifl >= 0, else it is invalid
      a.o = ifl + 1;
      a.v0 = -ifl;
      a.v1 = N - 2 - ifl;
    }
    a.w[0] = 1.0f;
    return true;
  }
  if (interp == IRP_INTERP_CUBIC) {
    // Keys' cubic convolution, a = -1/2: taps i0 - 1 .. i0 + 2 with weights
    // W(f + 1 - i); all four are non-zero for f > 0, only the one at i0 for
    // f = 0, and those must lie inside the frame
    a.o = ifl - 1;
    a.v0 = f > 0.0 ? 1 - ifl : -ifl;
    a.v1 = f > 0.0 ? N - 3 - ifl : N - 1 - ifl;
    for (int i = 0; i < 4; ++i) {
      const double t = std::fabs(f + 1.0 - i);
      double w = 0.0;
      if (t <= 1.0) w = 1.0 - 2.5 * t * t + 1.5 * t * t * t;
      else if (t < 2.0) w = -0.5 * (t - 1.0) * (t - 2.0) * (t - 2.0);
      a.w[i] = (float)w;
    }
    return true;
  }
  // taps with non-zero weight must lie inside: i0 >= 0, i0 + (f > 0) <= N - 1
  a.v0 = -ifl;
  a.v1 = N - 1 - ifl - (f > 0.0 ? 1 : 0);
  if (interp == IRP_INTERP_BILINEAR) {
    a.o = ifl;
    a.w[0] = (float)(1.0 - f);
    a.w[1] = (float)f;
  } else {  // cubic B-spline taps at i0 - 1 .. i0 + 2
    a.o = ifl - 1;
    for (int i = 0; i < 4; ++i) {
      const double t = std::fabs(f + 1.0 - i);
      double b = 0.0;
      if (t < 1.0) b = 2.0 / 3.0 - t * t + 0.5 * t * t * t;
      else if (t < 2.0) b = (2.0 - t) * (2.0 - t) * (2.0 - t) / 6.0;
      a.w[i] = (float)b;
    }
  }
  return true;
}

bool fill_geometry(FrameDesc& F, double dx, double dy, int W, int H, int interp) {
  Axis ax, ay;
  if (!split_axis(dx, W, interp, ax) || !split_axis(dy, H, interp, ay)) return false;
  F.ox = ax.o;
  F.oy = ay.o;
  F.fx = ax.f;
  F.fy = ay.f;
  F.vx0 = std::max(ax.v0, 0);
  F.vx1 = std::min(ax.v1, W - 1);
  F.vy0 = std::max(ay.v0, 0);
  F.vy1 = std::min(ay.v1, H - 1);
  for (int i = 0; i < 4; ++i) {
    F.wx[i] = ax.w[i];
    F.wy[i] = ay.w[i];
  }
  F.last_tap = (ax.f > 0.0f || (dx - std::floor(dx)) > 0.0 ? 1 : 0) |
               (ay.f > 0.0f || (dy - std::floor(dy)) > 0.0 ? 2 : 0);
  return true;
}

int stencil_of(irp_interp i) {
  switch (i) {
    case IRP_INTERP_NEAREST: return ST_NEAREST;
    case IRP_INTERP_BILINEAR: return ST_BILINEAR;
    case IRP_INTERP_CUBIC: return ST_CUBIC;
    default: return ST_BSPLINE;
  }
}

bool clip_ok(const irp_clip_params& c) {
  return std::isfinite(c.kappa_lo) && std::isfinite(c.kappa_hi) && c.kappa_lo > 0.0f &&
         c.kappa_hi > 0.0f && c.max_iter >= 0 && c.max_iter <= 1000 && (c.center == 0 || c.center == 1) &&
         (c.ddof == 0 || c.ddof == 1);
}

irp_status check_set(const irp_set& s) {
  if (!s.frames || s.W < 1 || s.H < 1 || s.n < 1) return IRP_ERR_INVALID_ARG;
  if (s.n > IRP_MAX_WIDE_FRAMES) return IRP_ERR_UNSUPPORTED;
  if ((int64_t)s.W * s.H > (int64_t)1 << 31) return IRP_ERR_UNSUPPORTED;
  if (s.raw_pitch < s.W || s.master_pitch < s.W) return IRP_ERR_INVALID_ARG;
  if (!s.dx || !s.dy || !s.exptime || !s.bias || !s.dark_rate || !s.flat) return IRP_ERR_INVALID_ARG;
  if (!s.mean_out && !s.median_out && !s.nkept_out && !s.stack_out) return IRP_ERR_INVALID_ARG;
  if ((s.mean_out || s.median_out || s.nkept_out || s.stack_out) && s.out_pitch < s.W)
    return IRP_ERR_INVALID_ARG;
  if (!aligned(s.bias, 4) || !aligned(s.dark_rate, 4) || !aligned(s.flat, 4) ||
      !aligned(s.mean_out, 4) || !aligned(s.median_out, 4) || !aligned(s.nkept_out, 2) ||
      !aligned(s.stack_out, 4) || !aligned(s.ready_flag, 4))
    return IRP_ERR_ALIGNMENT;
  if (s.mask && s.mask_pitch < s.W) return IRP_ERR_INVALID_ARG;
  if (!(s.saturation >= 0.0f) || std::isinf(s.saturation)) return IRP_ERR_INVALID_ARG;
  for (int k = 0; k < s.n; ++k) {
    if (!s.frames[k]) return IRP_ERR_INVALID_ARG;
    if (!aligned(s.frames[k], 2)) return IRP_ERR_ALIGNMENT;
    if (!std::isfinite(s.exptime[k]) || !std::isfinite(s.dx[k]) || !std::isfinite(s.dy[k]) ||
        std::fabs(s.dx[k]) > 1.0e9 || std::fabs(s.dy[k]) > 1.0e9)
      return IRP_ERR_INVALID_ARG;
  }
  return IRP_OK;
}

// ---------------------------------------------------------------------------
// Launch plan of irp_reduce_set.  Sets are grouped by register bucket of
// their frame count (one kernel instantiation each); within a group they are
// ordered by decreasing frame count, so that a persistent launch hands out
// the most expensive tiles first.
// ---------------------------------------------------------------------------
struct SubInfo {
  uint64_t dev_off;     // offset of this sub-plan image inside the workspace
  uint64_t img_off;     // offset of the image inside the plan file
  uint64_t bytes;       // image size
  uint64_t smem;        // dynamic shared memory of the reduce launch
  int32_t bucket, stencil, grid, pgrid;
  int32_t nitems, counter, nsets, nframes;
  int32_t nrows, ncolsegs, row_e, py;   // spline row / column passes, rows per warp
  int32_t norm_rb;                      // frame means: most row blocks of a set (0: none)
  int32_t tile_rows;                    // output rows per tile
};

struct PlanFile {
  uint32_t magic;
  int32_t nsub, interp, normalize_flat;
  int32_t nflat, persistent, nsets, ndeep;
  uint64_t ws_required;
  uint64_t flat_off;    // FrameStats[nflat] in the workspace
  uint64_t deep_off;    // CombineArgs[ndeep] in the plan file: the deep sets' combines
  uint64_t norm_off;    // FrameNorm records in the workspace (zeroed per call) ...
  uint64_t norm_bytes;  // ... and their size (0: no per-frame normalisation)
  SubInfo sub[kMaxSub];
};

struct FlatJob {  // follows PlanFile: one FP64 flat sum per set (normalize_flat)
  const float* flat;
  int64_t pitch;
  int32_t W, H;
};

struct Layout {
  size_t flat_off, plan_off, coef_off, total;
  std::vector<size_t> coef_frame_off;  // per set: offset of its first coefficient frame
  std::vector<size_t> crow_frame_off;  // per set: offset of its first row-pass frame
  std::vector<size_t> bad_frame_off;   // per set: offset of its first bad-pixel bit plane
  size_t norm_off = 0, norm_bytes = 0;
  std::vector<size_t> norm_user_off;   // per caller's set: its frames' FrameNorm records
  std::vector<size_t> stack_off;       // per deep set: its aligned stack (0: caller's)
};

// Sets deeper than the register buckets (IRP_MAX_FRAMES < n <=
// IRP_MAX_WIDE_FRAMES) are combined by groups of lanes.
// * Masked cubic-spline sets on the row pass with at most kWideTileMax
//   frames: the tile kernel's lane-group form, one kernel from the row-pass
//   coefficients like the shallower sets (a plain entry of its own bucket).
// * Other cubic-spline sets on the row + column passes, without a caller
//   stack, are reduced in two steps: the
//   column pass already leaves each frame's rows filtered along x on the
//   output grid, so the set only runs its prefilter, and the combine applies
//   the four vertical taps itself while it gathers the samples.
// * Otherwise chunks of at most kDeepChunk frames go through the fused kernel
//   as sets of their own that write the aligned FP32 stack and combine
//   nothing; the combine then reads the stack.  Chunks of 13 to 16 frames
//   share one register bucket, so a call adds one sub-plan per spline path
//   at most.
constexpr int kDeepChunk = 16;

struct DeepSet {
  int user;         // index in the caller's array
  int64_t spitch;   // stack row pitch (elements)
  bool own_stack;   // the stack lives in the workspace (no caller stack_out)
  bool rows;        // combined from the filtered spline rows (no stack)
};

struct PlanSets {
  std::vector<irp_set> sets;  // plain sets and the chunks of deep sets, in call order
  std::vector<int> deep_of;   // per entry: its deep set, or -1
  std::vector<int> k0;        // per entry: first frame of the chunk in its deep set
  std::vector<int> user_of;   // per entry: index of its set in the caller's array
  std::vector<DeepSet> deep;
  const irp_set* user;
  int interp = 0;
  bool onchip = false;  // spline_onchip: unmasked spline sets on the tile kernel
  int nsets() const { return (int)sets.size(); }
};

int64_t deep_stack_pitch(int W) { return (int64_t)align_up((size_t)W, 32); }

int spline_path(int W, int H);
bool tile_path(const PlanSets& ps, int i);



// A set deeper than the register buckets that the wide tile kernel reduces:
// masked cubic-spline sets on the row pass (the two-step path below has no
// bad-pixel footprint).  Unmasked ones keep the two-step path, measured
// faster on 180 x 1020^2 (2.24 ms against 4.9 to 5.8 ms for the tile form,
// which holds a tile's samples on chip at one or two CTAs per SM).
bool wide_tile_set(const irp_set& s, int interp) {
  return s.n > IRP_MAX_FRAMES && s.n <= kWideTileMax && interp == IRP_INTERP_SPLINE3 &&
         spline_path(s.W, s.H) && (s.mask || s.saturation > 0.0f);
}

// Bucket of a plan entry: the register bucket, or the wide tile kernel's.
int set_bucket(int n) { return n <= IRP_MAX_FRAMES ? reduce_bucket(n) : wide_tile_bucket(n); }

PlanSets expand_sets(const irp_set* sets, int nsets, int interp, bool onchip) {
  PlanSets ps;
  ps.user = sets;
  ps.interp = interp;
  ps.onchip = onchip;
  for (int i = 0; i < nsets; ++i) {
    const irp_set& s = sets[i];
    if (s.n <= IRP_MAX_FRAMES || wide_tile_set(s, interp)) {
      ps.sets.push_back(s);
      ps.user_of.push_back(i);
      ps.deep_of.push_back(-1);
      ps.k0.push_back(0);
      continue;
    }
    DeepSet d;
    d.user = i;
    d.rows = interp == IRP_INTERP_SPLINE3 && spline_path(s.W, s.H) && !s.stack_out;
    if (d.rows) {  // the whole set, prefilter only
      d.own_stack = false;
      d.spitch = 0;
      irp_set cs = s;
      cs.mean_out = nullptr;
      cs.median_out = nullptr;
      cs.nkept_out = nullptr;
      ps.sets.push_back(cs);
      ps.user_of.push_back(i);
      ps.deep_of.push_back((int)ps.deep.size());
      ps.k0.push_back(0);
      ps.deep.push_back(d);
      continue;
    }
    d.own_stack = s.stack_out == nullptr;
    d.spitch = d.own_stack ? deep_stack_pitch(s.W) : s.out_pitch;
    const int nch = (s.n + kDeepChunk - 1) / kDeepChunk;
    for (int c = 0; c < nch; ++c) {
      const int a = (int)((int64_t)c * s.n / nch), b = (int)((int64_t)(c + 1) * s.n / nch);
      irp_set cs = s;
      cs.frames = s.frames + a;
      cs.dx = s.dx + a;
      cs.dy = s.dy + a;
      cs.exptime = s.exptime + a;
      cs.n = b - a;
      cs.mean_out = nullptr;
      cs.median_out = nullptr;
      cs.nkept_out = nullptr;
      cs.stack_out = nullptr;  // placed in the stack by encode_plan
      cs.out_pitch = d.spitch;
      ps.sets.push_back(cs);
      ps.user_of.push_back(i);
      ps.deep_of.push_back((int)ps.deep.size());
      ps.k0.push_back(a);
    }
    ps.deep.push_back(d);
  }
  return ps;
}

// Spline prefilter of a set: row + column passes (1) or tiled (0).
int spline_path(int W, int H) {
  return (W >= kSplineMinSide && W <= kSplineMaxW && H >= kSplineMinSide) ? 1 : 0;
}

// A cubic-spline set on the row pass that the tile kernel reduces (not a
// deep set or one of its chunks).
// Unmasked sets take it when the caller asks for the on-chip form
// (spline_onchip); the row pass, column pass and vertical-tap reduction are
// faster (10 x 1024^2: 0.23 against 0.31 ms for 3 sets; 30 frames: 0.64
// against 1.34 ms) but move the row-pass and filtered frames through HBM.
bool tile_path(const PlanSets& ps, int i) {
  const irp_set& s = ps.sets[i];
  return ps.interp == IRP_INTERP_SPLINE3 && ps.deep_of[i] < 0 && spline_path(s.W, s.H) &&
         (ps.onchip || s.mask || s.saturation > 0.0f);
}
int64_t crow_pitch(int W) { return (int64_t)align_up((size_t)W, 4); }
// Bad-pixel bits of a masked spline frame: one word per 32 columns and row.
int64_t bad_pitch(int W) { return (W + 31) / 32; }
size_t bad_frame_bytes(int W, int H) {
  return align_up((size_t)H * (size_t)bad_pitch(W) * sizeof(uint32_t), kAlign);
}
size_t crow_frame_bytes(int W, int H) {
  return align_up((size_t)H * (size_t)crow_pitch(W) * sizeof(float), kAlign);
}

// Share of L2 a launch sequence keeps row-pass frames resident in.
constexpr size_t kL2Budget = (size_t)48 << 20;

// Spline coefficients are stored with a 2-sample mirrored border on every side.
int64_t coef_pitch(int W) { return (int64_t)align_up((size_t)W + 4, 4); }
size_t coef_frame_bytes(int W, int H) {
  return align_up((size_t)(H + 4) * (size_t)coef_pitch(W) * sizeof(float), kAlign);
}

// Sets are grouped by register bucket and, for the cubic spline, by the way
// their coefficients are formed (the two take different reduction kernels).
// Chunks of deep sets form groups of their own (no shared memory for
// samples), and whole deep sets that only run their prefilter another.
int group_key(const PlanSets& ps, int i, int interp) {
  const irp_set& s = ps.sets[i];
  const int b = set_bucket(s.n);
  const int key = interp == IRP_INTERP_SPLINE3
                      ? 4 * b + 2 * (tile_path(ps, i) ? 1 : 0) + spline_path(s.W, s.H)
                      : 4 * b;
  if (ps.deep_of[i] < 0) return key;
  return ps.deep[ps.deep_of[i]].rows ? 20000 : key + 10000;
}

void group_sets(const PlanSets& ps, int interp, std::vector<std::vector<int>>& groups) {
  const int nsets = ps.nsets();
  const irp_set* sets = ps.sets.data();
  std::vector<int> order(nsets);
  for (int i = 0; i < nsets; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const int ka = group_key(ps, a, interp), kb = group_key(ps, b, interp);
    return ka != kb ? ka > kb : sets[a].n > sets[b].n;
  });
  groups.clear();
  int cur = -1;
  for (int i : order) {
    const int key = group_key(ps, i, interp);
    if (key != cur) {
      groups.emplace_back();
      cur = key;
    }
    groups.back().push_back(i);
  }
}

Layout make_layout(const PlanSets& ps, const irp_reduce_params* p,
                   const std::vector<std::vector<int>>& groups) {
  const irp_set* sets = ps.sets.data();
  const int nsets = ps.nsets();
  Layout L;
  size_t off = sizeof(WsHeader);
  L.flat_off = off;
  off += align_up((size_t)nsets * sizeof(FrameStats), kAlign);
  // per-frame normalisation records, contiguous per caller's set (the chunks
  // of a deep set share its set's records, frame 0 first)
  L.norm_off = off;
  L.norm_user_off.clear();
  if (p->frame_norm) {
    int nuser = 0;
    for (int i = 0; i < nsets; ++i) nuser = std::max(nuser, ps.user_of[i] + 1);
    L.norm_user_off.assign(nuser, 0);
    for (int u = 0; u < nuser; ++u) {
      L.norm_user_off[u] = off;
      off += (size_t)ps.user[u].n * sizeof(FrameNorm);
    }
    off = align_up(off, kAlign);
  }
  L.norm_bytes = off - L.norm_off;
  L.plan_off = off;
  for (const auto& g : groups) {
    int nf = 0;
    for (int i : g) nf += sets[i].n;
    off += align_up(plan_total_bytes((int)g.size(), nf), kAlign);
  }
  L.coef_off = off;
  L.coef_frame_off.assign(nsets, 0);
  L.crow_frame_off.assign(nsets, 0);
  L.bad_frame_off.assign(nsets, 0);
  if (p->interp == IRP_INTERP_SPLINE3) {
    for (int i = 0; i < nsets; ++i) {
      const irp_set& s = sets[i];
      // sets on the tile kernel need no filtered frames, only the row pass's
      if (!tile_path(ps, i)) {
        L.coef_frame_off[i] = off;
        off += (size_t)s.n * coef_frame_bytes(s.W, s.H);
      }
      if (spline_path(s.W, s.H)) {
        L.crow_frame_off[i] = off;
        off += (size_t)s.n * crow_frame_bytes(s.W, s.H);
        if (tile_path(ps, i) && (s.mask || s.saturation > 0.0f)) {
          L.bad_frame_off[i] = off;
          off += (size_t)s.n * bad_frame_bytes(s.W, s.H);
        }
      }
    }
  }
  L.stack_off.assign(ps.deep.size(), 0);
  for (size_t d = 0; d < ps.deep.size(); ++d) {
    if (!ps.deep[d].own_stack) continue;
    const irp_set& u = ps.user[ps.deep[d].user];
    L.stack_off[d] = off;
    off += align_up((size_t)u.n * u.H * ps.deep[d].spitch * sizeof(float), kAlign);
  }
  L.total = off;
  return L;
}

irp_status check_params(const irp_set* sets, int nsets, const irp_reduce_params* p) {
  if (!sets || !p || nsets < 1) return IRP_ERR_INVALID_ARG;
  if (p->interp < IRP_INTERP_NEAREST || p->interp > IRP_INTERP_CUBIC) return IRP_ERR_INVALID_ARG;
  if (!clip_ok(p->clip)) return IRP_ERR_INVALID_ARG;
  if (p->max_ctas < 0 || p->wait_spin_limit < 0 || p->rows_per_warp < 0) return IRP_ERR_INVALID_ARG;
  if (p->frame_norm < 0 || p->frame_norm > 2) return IRP_ERR_INVALID_ARG;
  if (p->spline_onchip < 0 || p->spline_onchip > 1) return IRP_ERR_INVALID_ARG;
  for (int i = 0; i < nsets; ++i) {
    irp_status st = check_set(sets[i]);
    if (st != IRP_OK) return st;
    // with the cubic spline, bad-pixel masking is built for the sets the tile
    // kernel reduces (34 <= W <= 8192, H >= 34, at most kWideTileMax frames)
    if (p->interp == IRP_INTERP_SPLINE3 && (sets[i].mask || sets[i].saturation > 0.0f) &&
        !(spline_path(sets[i].W, sets[i].H) && sets[i].n <= kWideTileMax))
      return IRP_ERR_UNSUPPORTED;
  }
  std::vector<std::vector<int>> groups;
  group_sets(expand_sets(sets, nsets, p->interp, p->spline_onchip != 0), p->interp, groups);
  if ((int)groups.size() > kMaxSub) return IRP_ERR_UNSUPPORTED;
  return IRP_OK;
}

// Device count of SMs, cached per process.
int sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 1;
  }
  return sms;
}

size_t deep_jobs_offset(int nsets) {
  return align_up(sizeof(PlanFile) + (size_t)nsets * sizeof(FlatJob), 64);
}

size_t plan_images_offset(const PlanSets& ps) {
  return align_up(deep_jobs_offset(ps.nsets()) + ps.deep.size() * sizeof(CombineArgs), 64);
}

size_t plan_file_bytes(const PlanSets& ps, const irp_reduce_params* p) {
  const irp_set* sets = ps.sets.data();
  std::vector<std::vector<int>> groups;
  group_sets(ps, p->interp, groups);
  size_t off = plan_images_offset(ps);
  for (const auto& g : groups) {
    int nf = 0;
    for (int i : g) nf += sets[i].n;
    off += align_up(plan_total_bytes((int)g.size(), nf), 64);
  }
  (void)p;
  return off;
}

// Encodes the plan file.  Needs the workspace address (descriptors point into
// it) but touches neither the device nor the workspace contents.
irp_status encode_plan(const PlanSets& ps, const irp_reduce_params* p, uint8_t* buf,
                       size_t buf_bytes, uint8_t* ws, size_t ws_bytes) {
  const irp_set* sets = ps.sets.data();
  const int nsets = ps.nsets();
  std::vector<std::vector<int>> groups;
  group_sets(ps, p->interp, groups);
  const Layout L = make_layout(ps, p, groups);
  if (!ws || !aligned(ws, kAlign)) return IRP_ERR_WORKSPACE;
  if (ws_bytes < L.total) return IRP_ERR_WORKSPACE;
  const size_t file_bytes = plan_file_bytes(ps, p);
  if (buf_bytes < file_bytes) return IRP_ERR_INVALID_ARG;
  std::memset(buf, 0, file_bytes);
  PlanFile* pf = (PlanFile*)buf;
  pf->magic = kPlanMagic;
  pf->nsub = (int)groups.size();
  pf->interp = p->interp;
  pf->normalize_flat = p->normalize_flat ? 1 : 0;
  pf->nflat = p->normalize_flat ? nsets : 0;
  pf->persistent = p->persistent ? 1 : 0;
  pf->ws_required = L.total;
  pf->flat_off = L.flat_off;
  pf->nsets = nsets;
  pf->ndeep = (int)ps.deep.size();
  pf->deep_off = deep_jobs_offset(nsets);
  pf->norm_off = L.norm_off;
  pf->norm_bytes = L.norm_bytes;
  // the deep sets' stacks and their lane-group combines
  std::vector<float*> stack_base(ps.deep.size());
  CombineArgs* dj = (CombineArgs*)(buf + pf->deep_off);
  for (size_t d = 0; d < ps.deep.size(); ++d) {
    const irp_set& u = ps.user[ps.deep[d].user];
    stack_base[d] = ps.deep[d].own_stack ? (float*)(ws + L.stack_off[d]) : u.stack_out;
    CombineArgs& a = dj[d];
    a.stack = ps.deep[d].rows ? nullptr : stack_base[d];  // rows: frames set below
    a.pitch = ps.deep[d].spitch;
    a.fstride = (int64_t)u.H * ps.deep[d].spitch;
    a.W = u.W;
    a.H = u.H;
    a.n = u.n;
    a.clip = ClipArgs{p->clip.kappa_lo, p->clip.kappa_hi, p->clip.max_iter, p->clip.center,
                      p->clip.ddof};
    a.mean_out = u.mean_out;
    a.median_out = u.median_out;
    a.nkept_out = u.nkept_out;
    a.out_pitch = u.out_pitch;
    // samples formed from filtered rows in the combine take the frames'
    // normalisation there; a stack already holds normalised samples
    a.frame_norm = (ps.deep[d].rows && p->frame_norm) ? 1 : 0;
  }
  FlatJob* fj = (FlatJob*)(buf + sizeof(PlanFile));
  for (int i = 0; i < nsets; ++i) {
    fj[i].flat = sets[i].flat;
    fj[i].pitch = sets[i].master_pitch;
    fj[i].W = sets[i].W;
    fj[i].H = sets[i].H;
  }
  const int stencil = stencil_of(p->interp);
  const int taps = (stencil == ST_BSPLINE || stencil == ST_CUBIC) ? 4 : (stencil == ST_BILINEAR ? 2 : 1);
  WsHeader* wsh = (WsHeader*)ws;
  size_t img_off = plan_images_offset(ps);
  size_t dev_off = L.plan_off;
  for (int gi = 0; gi < (int)groups.size(); ++gi) {
    const auto& g = groups[gi];
    int nf = 0, max_n = 0, mwin_f4 = 0;  // mwin_f4: the largest master window (float4 entries)
    for (int i : g) {
      nf += sets[i].n;
      max_n = std::max(max_n, sets[i].n);
    }
    const int bucket = set_bucket(max_n);
    const bool stack_only = ps.deep_of[g[0]] >= 0;  // the group holds deep-set chunks
    const bool pre_only = stack_only && ps.deep[ps.deep_of[g[0]]].rows;  // ... or whole sets
    // the group's reduction stencil: spline sets on the row + column passes
    // arrive horizontally filtered and take the vertical taps only
    const bool spline = stencil == ST_BSPLINE;
    const bool gpath = spline && spline_path(sets[g[0]].W, sets[g[0]].H);
    const bool gtile = gpath && tile_path(ps, g[0]);  // the tile kernel (no column pass)
    const int gstencil = gtile ? ST_BSPLINE_T : (gpath ? ST_BSPLINE_V : stencil);
    const int TWc = tile_cols(gstencil);
    // rows per warp: the caller's choice, else the bucket's default, unless the
    // group's tiles at the default would give fewer than two CTAs per SM; the
    // bucket's shorter tiles (where the other choice is shorter) then spread
    // the group further
    int py = rows_per_warp(bucket, gstencil, p->rows_per_warp);
    if (p->rows_per_warp == 0 && rows_per_warp_alt(bucket, gstencil) < py) {
      int64_t tiles = 0;
      for (int i : g)
        tiles += (int64_t)((sets[i].W + TWc - 1) / TWc) *
                 ((sets[i].H + tile_rows(bucket, py) - 1) / tile_rows(bucket, py));
      if (tiles < 2 * (int64_t)sm_count()) py = rows_per_warp_alt(bucket, gstencil);
    }
    const int THr = gtile ? spline_tile_rows(bucket, max_n) : tile_rows(bucket, py);
    // prefilter work items: tiles x frame groups, enough groups to fill the GPU twice
    int pgroups = 1;
    if (stencil == ST_BSPLINE) {
      int ptiles = 0;
      for (int i : g)
        ptiles += ((sets[i].W + kPrefTile - 1) / kPrefTile) * ((sets[i].H + kPrefTile - 1) / kPrefTile);
      pgroups = std::max(1, std::min(max_n, (2 * sm_count() + ptiles - 1) / std::max(ptiles, 1)));
    }
    uint8_t* img = buf + img_off;
    PlanHeader* h = (PlanHeader*)img;
    SetDesc* sd = (SetDesc*)(img + plan_sets_offset());
    FrameDesc* fd = (FrameDesc*)(img + plan_frames_offset((int)g.size()));
    int frame0 = 0, tile0 = 0, ptile0 = 0, nrows = 0, ncolsegs = 0, row_e = 32, norm_rb = 0;
    for (int si : g)  // row-pass width: 32 columns per lane, 64 when a frame is wider than 1024
      if (stencil == ST_BSPLINE && spline_path(sets[si].W, sets[si].H) && sets[si].W > 1024)
        row_e = 64;
    for (int si = 0; si < (int)g.size(); ++si) {
      const irp_set& s = sets[g[si]];
      SetDesc& S = sd[si];
      S.W = s.W;
      S.H = s.H;
      S.n = s.n;
      S.frame0 = frame0;
      S.src_pitch = s.raw_pitch;
      S.coef_pitch = stencil == ST_BSPLINE ? coef_pitch(s.W) : 0;
      S.bias = s.bias;
      S.dark = s.dark_rate;
      S.flat = s.flat;
      S.master_pitch = s.master_pitch;
      S.flat_sum = p->normalize_flat
                       ? (const double*)(ws + L.flat_off + (size_t)g[si] * sizeof(FrameStats))
                       : nullptr;
      S.mean_out = s.mean_out;
      S.median_out = s.median_out;
      S.nkept_out = s.nkept_out;
      S.stack_out = s.stack_out;
      S.out_pitch = s.out_pitch;
      if (ps.deep_of[g[si]] >= 0) {
        const int d = ps.deep_of[g[si]];
        S.stack_only = 1;
        if (ps.deep[d].rows) {
          // the combine reads the set's frame table from this sub-plan's image
          CombineArgs& a = dj[d];
          a.frames = (const FrameDesc*)(ws + dev_off + plan_frames_offset((int)g.size())) +
                     frame0;
          a.coef_pitch = coef_pitch(s.W);
        } else {
          S.stack_out = stack_base[d] + (int64_t)ps.k0[g[si]] * s.H * ps.deep[d].spitch;
        }
      }
      S.tiles_x = (s.W + TWc - 1) / TWc;
      S.tiles_y = (s.H + THr - 1) / THr;
      S.tile0 = tile0;
      if (!pre_only) tile0 += S.tiles_x * S.tiles_y;  // prefilter-only sets have no tiles
      S.ptiles_x = (s.W + kPrefTile - 1) / kPrefTile;
      S.ptiles_y = (s.H + kPrefTile - 1) / kPrefTile;
      S.ptile0 = ptile0;
      S.pframes = std::max(1, (s.n + pgroups - 1) / pgroups);
      if (stencil == ST_BSPLINE && !spline_path(s.W, s.H))
        ptile0 += S.ptiles_x * S.ptiles_y * ((s.n + S.pframes - 1) / S.pframes);
      S.ready_flag = s.ready_flag;
      S.ready_value = s.ready_value;
      S.mflags = (aligned(s.bias, 16) && aligned(s.dark_rate, 16) && aligned(s.flat, 16) &&
                  s.master_pitch % 4 == 0) ? 1 : 0;
      S.spath = stencil == ST_BSPLINE ? spline_path(s.W, s.H) : 0;
      S.mask = s.mask;
      S.mask_pitch = s.mask ? s.mask_pitch : 0;
      S.saturation = s.saturation > 0.0f ? s.saturation : INFINITY;
      S.masked = (s.mask || s.saturation > 0.0f) ? 1 : 0;
      S.crow_pitch = S.spath ? crow_pitch(s.W) : 0;
      S.row0 = nrows;
      S.colseg0 = ncolsegs;
      S.bad_pitch = bad_pitch(s.W);
      const int user = ps.user_of[g[si]];
      S.norm_ref = p->frame_norm ? (const FrameNorm*)(ws + L.norm_user_off[user]) : nullptr;
      if (p->frame_norm) {
        const int R = stats_rows(s.W, s.H);
        norm_rb = std::max(norm_rb, (s.H + R - 1) / R);
      }
      if (S.spath) {
        // frames per row-pass work item (each work item reads its block's
        // masters once; smaller groups measured slower on 10 x 1024^2 sets:
        // more CTAs than one wave)
        const int nrb = (s.H + row_block(row_e) - 1) / row_block(row_e);
        S.rgroup = std::min(kRowGroup, s.n);
        nrows += ((s.n + S.rgroup - 1) / S.rgroup) * row_segments(s.W) * nrb;
        if (!gtile) ncolsegs += s.n * ((s.W + 28) / 29) * ((s.H + kColRows - 1) / kColRows);
      }
      // premerged master window {bias + dark*t, rf}: raw sources of one
      // exposure time without a bad-pixel mask or saturation level
      bool one_t = true;
      for (int k = 1; k < s.n; ++k) one_t = one_t && s.exptime[k] == s.exptime[0];
      if (stencil != ST_BSPLINE && !S.masked && one_t) S.mflags |= 2;
      int oxmin = INT32_MAX, oxmax = INT32_MIN, oymin = INT32_MAX, oymax = INT32_MIN;
      for (int k = 0; k < s.n; ++k) {
        FrameDesc& F = fd[frame0 + k];
        if (!fill_geometry(F, s.dx[k], s.dy[k], s.W, s.H, p->interp)) return IRP_ERR_INVALID_ARG;
        F.src = s.frames[k];
        F.flags = (aligned(s.frames[k], 16) && s.raw_pitch % 8 == 0) ? 1 : 0;
        F.flags |= (aligned(s.frames[k], 8) && s.raw_pitch % 4 == 0) ? 2 : 0;
        F.t = s.exptime[k];
        F.scale = 1.0f;
        F.offset = 0.0f;
        F.coef = stencil == ST_BSPLINE
                     ? (float*)(ws + L.coef_frame_off[g[si]] + (size_t)k * coef_frame_bytes(s.W, s.H))
                     : nullptr;
        F.crow = (stencil == ST_BSPLINE && spline_path(s.W, s.H))
                     ? (float*)(ws + L.crow_frame_off[g[si]] + (size_t)k * crow_frame_bytes(s.W, s.H))
                     : nullptr;
        F.bad = L.bad_frame_off[g[si]]
                    ? (const uint32_t*)(ws + L.bad_frame_off[g[si]] +
                                        (size_t)k * bad_frame_bytes(s.W, s.H))
                    : nullptr;
        if (gtile) F.coef = nullptr;
        F.norm = p->frame_norm ? (FrameNorm*)(ws + L.norm_user_off[user]) + ps.k0[g[si]] + k
                               : nullptr;
        oxmin = std::min(oxmin, F.ox);
        oxmax = std::max(oxmax, F.ox);
        oymin = std::min(oymin, F.oy);
        oymax = std::max(oymax, F.oy);
      }
      // master union window over all frames' taps ({bias, dark, 1/flat, mask},
      // 16 B each, or 12 B staged and premerged), kept unless the offsets are
      // so spread that it would exceed 64 KB
      const int mw = 32 + (oxmax - oxmin), mh = THr + (oymax - oymin) + taps - 1;
      if (stencil != ST_BSPLINE && mw * mh <= kMaxWindowPx) {
        S.mwin_w = mw;
        S.mwin_h = mh;
        S.mox = oxmin;
        S.moy = oymin;
        mwin_f4 = std::max(mwin_f4, master_window_f4(mw, mh, (S.mflags & 2) != 0));
      }
      frame0 += s.n;
    }
    h->nsets = (int)g.size();
    h->nframes = nf;
    h->nitems = tile0;
    h->npitems = ptile0;
    h->nrows = nrows;
    h->ncolsegs = ncolsegs;
    h->stencil = gstencil;
    h->max_n = max_n;
    h->persistent = p->persistent ? 1 : 0;
    h->spin_limit = p->wait_spin_limit > 0 ? p->wait_spin_limit : kDefaultSpin;
    h->src = stencil == ST_BSPLINE ? SRC_F32 : SRC_RAW;
    h->kappa_lo = p->clip.kappa_lo;
    h->kappa_hi = p->clip.kappa_hi;
    h->max_iter = p->clip.max_iter;
    h->center = p->clip.center;
    h->ddof = p->clip.ddof;
    h->frame_norm = p->frame_norm;
    h->smem_samples = stack_only ? 0 : max_n * THr * 32;
    h->smem_master = mwin_f4;
    h->status = &wsh->status;
    h->counter = &wsh->counters[gi];
    SubInfo& si = pf->sub[gi];
    si.dev_off = dev_off;
    si.img_off = img_off;
    si.bytes = plan_total_bytes((int)g.size(), nf);
    si.bucket = bucket;
    si.py = py;
    si.stencil = gstencil;
    si.smem = gtile ? spline_tile_smem_bytes(bucket, max_n)
                    : reduce_smem_bytes(spline ? SRC_F32 : SRC_RAW, gstencil, py, max_n, mwin_f4) -
                          (stack_only ? (size_t)max_n * THr * 32 * sizeof(float) : 0);
    si.nitems = tile0;
    si.counter = gi;
    si.nsets = (int)g.size();
    si.nframes = nf;
    si.pgrid = stencil == ST_BSPLINE ? ptile0 : 0;
    si.nrows = nrows;
    si.ncolsegs = ncolsegs;
    si.row_e = row_e;
    si.norm_rb = norm_rb;
    si.tile_rows = THr;
    if (si.smem > 227 * 1024 - 1024) return IRP_ERR_UNSUPPORTED;  // opt-in limit less static smem
    if (p->persistent && !gtile) {
      const int occ = reduce_occupancy(si.bucket, si.py, gstencil, si.smem);
      int g_ctas = p->max_ctas > 0 ? p->max_ctas : occ * sm_count();
      si.grid = std::max(1, std::min(g_ctas, tile0));
    } else {
      si.grid = tile0;
    }
    img_off += align_up(si.bytes, 64);
    dev_off += align_up(si.bytes, kAlign);
  }
  return IRP_OK;
}

// Row-pass coefficients kept resident in L2 between the row pass and the
// tile kernel (L2 holds about 126 MB; the raw frames, masters and outputs
// stream through beside them).

// A sub-plan of cubic-spline sets reduced by the tile kernel.  Its sets go in
// order, in runs of consecutive sets whose row-pass coefficients fit within
// kL2Budget together: the row pass of a run, then the tile kernel of the run,
// so that the tile kernel reads the coefficients from L2, and then the run's
// coefficients are dropped from L2 without being written back.  A set larger
// than the budget goes in stripes of rows: the row pass of a stripe, the
// tiles whose rows (with the recursions' warm-up rows) are complete, and the
// coefficient rows no later tile reads dropped.
irp_status run_tile_subplan(const uint8_t* buf, const SubInfo& si, const InlinePlan* inl,
                            const void* dev_plan, cudaStream_t s) {
  const uint8_t* img = buf + si.img_off;
  const SetDesc* sd = (const SetDesc*)(img + plan_sets_offset());
  const FrameDesc* fd = (const FrameDesc*)(img + plan_frames_offset(si.nsets));
  const int RB = row_block(si.row_e);
  const int TH = si.tile_rows;
  auto set_bytes = [&](int j) {  // row-pass frames, then bad-pixel planes, contiguous
    const SetDesc& S = sd[j];
    return (size_t)S.n * (crow_frame_bytes(S.W, S.H) +
                          (fd[S.frame0].bad ? bad_frame_bytes(S.W, S.H) : 0));
  };
  cudaError_t e = cudaSuccess;
  auto rows = [&](int i0, int count) {
    if (e != cudaSuccess || count <= 0) return;
    TraceScope tr(IRP_KERNEL_PREFILTER, s);
    e = launch_spline_rows(si.row_e, inl, dev_plan, i0, count, s);
  };
  auto tiles = [&](int i0, int count) {
    if (e != cudaSuccess || count <= 0) return;
    TraceScope tr(IRP_KERNEL_REDUCE, s);
    e = launch_spline_tile(si.bucket, si.tile_rows, inl, dev_plan, i0, count, si.smem, s, false);
  };
  auto discard = [&](const void* p, size_t bytes, int count, size_t stride) {
    if (e != cudaSuccess || bytes == 0) return;
    TraceScope tr(IRP_KERNEL_PREFILTER, s);
    e = launch_discard_l2(p, bytes, count, stride, s);
  };
  for (int a = 0; a < si.nsets && e == cudaSuccess;) {
    size_t bytes = set_bytes(a);
    int b = a + 1;
    while (b < si.nsets && bytes + set_bytes(b) <= kL2Budget) bytes += set_bytes(b++);
    if (b == a + 1 && bytes > kL2Budget) {
      // one set in stripes of rows
      const SetDesc& S = sd[a];
      // row-pass work items per row block: frame groups x row segments
      const int ngroups = (S.n + S.rgroup - 1) / S.rgroup * row_segments(S.W);
      const int nrb = (S.H + RB - 1) / RB;
      int oymin = INT32_MAX, oymax = INT32_MIN;
      for (int k = 0; k < S.n; ++k) {
        oymin = std::min(oymin, fd[S.frame0 + k].oy);
        oymax = std::max(oymax, fd[S.frame0 + k].oy);
      }
      const size_t row_bytes = (size_t)S.n * (size_t)S.crow_pitch * sizeof(float);
      int R = (int)std::min<size_t>((size_t)S.H, kL2Budget / 2 / row_bytes);
      R = std::max(TH, R / TH * TH);
      int done_rows = 0, done_out = 0, dead = 0;
      while (done_out < S.H && e == cudaSuccess) {
        const int target = std::min(S.H, done_rows + R);
        const int rb0 = done_rows / RB, rb1 = target >= S.H ? nrb : target / RB;
        rows(S.row0 + rb0 * ngroups, (rb1 - rb0) * ngroups);
        done_rows = rb1 >= nrb ? S.H : rb1 * RB;
        // output rows whose taps and warm-up rows are all on hand
        int out = done_rows >= S.H ? S.H : (done_rows - 3 - 16 - oymax) / TH * TH;
        out = std::max(out, done_out);
        if (out > done_out) {
          const int ty0 = done_out / TH, ty1 = (out + TH - 1) / TH;
          tiles(S.tile0 + ty0 * S.tiles_x, (ty1 - ty0) * S.tiles_x);
          done_out = out;
        }
        // coefficient rows no later tile reads (the first later tile starts
        // at done_out and reads from done_out + oymin - 16 on)
        const int nd = std::min(done_rows, std::max(0, done_out + oymin - 16));
        if (nd > dead && done_out < S.H) {
          discard((const uint8_t*)fd[S.frame0].crow + (size_t)dead * S.crow_pitch * 4,
                  (size_t)(nd - dead) * S.crow_pitch * 4, S.n, crow_frame_bytes(S.W, S.H));
          dead = nd;
        }
      }
      discard(fd[S.frame0].crow, set_bytes(a), 1, 0);
    } else {
      const int r0 = sd[a].row0, r1 = b < si.nsets ? sd[b].row0 : si.nrows;
      const int t0 = sd[a].tile0, t1 = b < si.nsets ? sd[b].tile0 : si.nitems;
      rows(r0, r1 - r0);
      tiles(t0, t1 - t0);
      for (int j = a; j < b; ++j) discard(fd[sd[j].frame0].crow, set_bytes(j), 1, 0);
    }
    a = b;
  }
  return cuda_status(e);
}

// Launches an encoded plan.  ``upload``: copy the sub-plan images into the
// workspace (else every sub-plan is passed by value as a kernel parameter).
irp_status run_plan(const uint8_t* buf, uint8_t* ws, size_t ws_bytes, cudaStream_t s, bool upload) {
  const PlanFile* pf = (const PlanFile*)buf;
  if (pf->magic != kPlanMagic || pf->nsub < 1 || pf->nsub > kMaxSub) return IRP_ERR_INVALID_ARG;
  if (!ws || !aligned(ws, kAlign) || ws_bytes < pf->ws_required) return IRP_ERR_WORKSPACE;
  WsHeader* wsh = (WsHeader*)ws;
  cudaError_t e = cudaSuccess;
  if (upload) {
    // the images are contiguous in the file and in the workspace up to padding;
    // copy them one by one (one copy per sub-plan)
    for (int i = 0; i < pf->nsub && e == cudaSuccess; ++i)
      e = cudaMemcpyAsync(ws + pf->sub[i].dev_off, buf + pf->sub[i].img_off, pf->sub[i].bytes,
                          cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return note_cuda(e);
  }
  if (pf->nflat > 0) {
    FrameStats* st = (FrameStats*)(ws + pf->flat_off);
    const FlatJob* fj = (const FlatJob*)(buf + sizeof(PlanFile));
    TraceScope tr(IRP_KERNEL_STATS, s);
    e = launch_stats_init(st, pf->nflat, s);
    for (int i = 0; i < pf->nflat && e == cudaSuccess; ++i)
      e = launch_stats_frames(fj[i].flat, fj[i].pitch, 0, fj[i].W, fj[i].H, 1, false, nullptr,
                              nullptr, nullptr, nullptr, nullptr, st + i, s);
    if (e != cudaSuccess) return note_cuda(e);
  }
  if (pf->norm_bytes > 0) {  // per-frame normalisation: the sums start at zero
    e = cudaMemsetAsync(ws + pf->norm_off, 0, pf->norm_bytes, s);
    if (e != cudaSuccess) return note_cuda(e);
  }
  for (int i = 0; i < pf->nsub; ++i) {
    const SubInfo& si = pf->sub[i];
    const void* dev_plan = upload ? (const void*)(ws + si.dev_off) : nullptr;
    InlinePlan inl;
    if (!upload) {
      // repack the image (header, sets, frames) into the fixed inline layout
      const uint8_t* img = buf + si.img_off;
      std::memset(&inl, 0, sizeof(inl));
      std::memcpy(&inl.h, img, sizeof(PlanHeader));
      std::memcpy(inl.sets, img + plan_sets_offset(), (size_t)si.nsets * sizeof(SetDesc));
      std::memcpy(inl.frames, img + plan_frames_offset(si.nsets), (size_t)si.nframes * sizeof(FrameDesc));
    } else {
      std::memset(&inl.h, 0, sizeof(PlanHeader));
    }
    if (si.norm_rb > 0) {  // the frames' mean levels, then their normalisation factors
      TraceScope tr(IRP_KERNEL_STATS, s);
      e = launch_frame_norm(&inl, dev_plan, si.nframes, si.norm_rb, s);
      if (e != cudaSuccess) return note_cuda(e);
    }
    if (si.stencil == ST_BSPLINE_T) {  // row pass and tile kernel, interleaved
      const irp_status st = run_tile_subplan(buf, si, &inl, dev_plan, s);
      if (st != IRP_OK) return st;
      continue;
    }
    if (si.pgrid > 0 || si.nrows > 0) {
      TraceScope tr(IRP_KERNEL_PREFILTER, s);
      if (si.pgrid > 0) e = launch_prefilter_raw(&inl, dev_plan, si.pgrid, s);
      if (e == cudaSuccess && si.nrows > 0)
        e = launch_spline_rows(si.row_e, &inl, dev_plan, 0, si.nrows, s);
      if (e == cudaSuccess && si.ncolsegs > 0)
        e = launch_spline_cols(&inl, dev_plan, 0, si.ncolsegs, s);
      if (e != cudaSuccess) return note_cuda(e);
    }
    if (si.nitems == 0) continue;  // prefilter-only sub-plan (deep spline sets)
    if (pf->persistent) {
      e = cudaMemsetAsync(&wsh->counters[si.counter], 0, sizeof(uint32_t), s);
      if (e != cudaSuccess) return note_cuda(e);
    }
    {
      TraceScope tr(IRP_KERNEL_REDUCE, s);
      e = launch_reduce(si.bucket, si.py, si.stencil, &inl, dev_plan, si.grid, si.smem, s);
    }
    if (e != cudaSuccess) return note_cuda(e);
  }
  // deep sets: their stacks are complete in stream order
  const CombineArgs* dj = (const CombineArgs*)(buf + pf->deep_off);
  for (int d = 0; d < pf->ndeep; ++d) {
    TraceScope tr(IRP_KERNEL_COMBINE, s);
    e = launch_combine_wide(dj[d], false, s);
    if (e != cudaSuccess) return note_cuda(e);
  }
  return IRP_OK;
}

// Copy streams of irp_reduce_set_host, one pair per device (created on first
// use and kept for the process), and the events that order them.
struct HostPipe {
  std::mutex mu;
  cudaStream_t up = nullptr, down = nullptr;
  std::vector<cudaEvent_t> ev;
};

cudaError_t host_pipe(HostPipe** out) {
  constexpr int kMaxDevices = 64;
  static std::mutex mu;
  static HostPipe pipes[kMaxDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  HostPipe& hp = pipes[dev];
  if (!hp.up) e = cudaStreamCreateWithFlags(&hp.up, cudaStreamNonBlocking);
  if (e == cudaSuccess && !hp.down) e = cudaStreamCreateWithFlags(&hp.down, cudaStreamNonBlocking);
  *out = &hp;
  return e;
}

// At least `count` events in the pipe (caller holds hp->mu).
cudaError_t host_pipe_events(HostPipe* hp, int count) {
  while ((int)hp->ev.size() < count) {
    cudaEvent_t ev = nullptr;
    const cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    hp->ev.push_back(ev);
  }
  return cudaSuccess;
}

bool plan_fits_inline(const uint8_t* buf) {
  const PlanFile* pf = (const PlanFile*)buf;
  if (pf->ndeep > 0) return false;  // deep combines read frame tables in the workspace
  for (int i = 0; i < pf->nsub; ++i)
    if (pf->sub[i].nsets > kMaxInlineSets || pf->sub[i].nframes > kMaxInlineFrames) return false;
  return true;
}

}  // namespace

extern "C" {

int irp_version(void) { return IRP_VERSION; }

const char* irp_last_cuda_error(void) { return g_last_cuda_error; }

const char* irp_status_string(irp_status s) {
  switch (s) {
    case IRP_OK: return "ok";
    case IRP_ERR_INVALID_ARG: return "invalid argument";
    case IRP_ERR_ALIGNMENT: return "misaligned buffer";
    case IRP_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case IRP_ERR_UNSUPPORTED: return "unsupported request";
    case IRP_ERR_BAD_MASTER: return "flat master value not finite or not positive";
    case IRP_ERR_CUDA: return "CUDA runtime error";
    case IRP_ERR_TIMEOUT: return "bounded device wait timed out";
    case IRP_ERR_BAD_STATISTIC: return "a frame's mean level is zero or not finite";
  }
  return "unknown status";
}

int irp_device_sm_count(void) { return sm_count(); }

void irp_profile_enable(int on) { tracer().on = on != 0; }

int irp_profile_read(double* ms_out, int64_t* launches_out, int max_kinds) {
  const int kinds = std::min(max_kinds, (int)IRP_KERNEL_KINDS);
  for (int k = 0; k < kinds; ++k) {
    if (ms_out) ms_out[k] = 0.0;
    if (launches_out) launches_out[k] = 0;
  }
  Tracer& t = tracer();
  for (const TraceRec& r : t.recs) {
    float ms = 0.0f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess &&
        r.kind < kinds) {
      if (ms_out) ms_out[r.kind] += ms;
      if (launches_out) launches_out[r.kind] += 1;
    }
    t.pool.push_back(r.a);
    t.pool.push_back(r.b);
  }
  t.recs.clear();
  return kinds;
}

size_t irp_workspace_size(const irp_set* sets, int nsets, const irp_reduce_params* p) {
  if (check_params(sets, nsets, p) != IRP_OK) return 0;
  const PlanSets ps = expand_sets(sets, nsets, p->interp, p->spline_onchip != 0);
  std::vector<std::vector<int>> groups;
  group_sets(ps, p->interp, groups);
  return make_layout(ps, p, groups).total;
}

size_t irp_plan_bytes(const irp_set* sets, int nsets, const irp_reduce_params* p) {
  if (check_params(sets, nsets, p) != IRP_OK) return 0;
  return plan_file_bytes(expand_sets(sets, nsets, p->interp, p->spline_onchip != 0), p);
}

irp_status irp_plan_encode(const irp_set* sets, int nsets, const irp_reduce_params* p,
                           void* plan_host, size_t plan_bytes, void* workspace, size_t ws_bytes) {
  irp_status st = check_params(sets, nsets, p);
  if (st != IRP_OK) return st;
  if (!plan_host) return IRP_ERR_INVALID_ARG;
  return encode_plan(expand_sets(sets, nsets, p->interp, p->spline_onchip != 0), p, (uint8_t*)plan_host, plan_bytes,
                     (uint8_t*)workspace, ws_bytes);
}

irp_status irp_plan_launch(const void* plan_host, size_t plan_bytes, void* workspace,
                           size_t ws_bytes, void* stream) {
  if (!plan_host || plan_bytes < sizeof(PlanFile)) return IRP_ERR_INVALID_ARG;
  return run_plan((const uint8_t*)plan_host, (uint8_t*)workspace, ws_bytes, (cudaStream_t)stream,
                  true);
}

irp_status irp_reduce_set(const irp_set* sets, int nsets, const irp_reduce_params* p,
                          void* workspace, size_t ws_bytes, void* stream) {
  irp_status st = check_params(sets, nsets, p);
  if (st != IRP_OK) return st;
  const PlanSets ps = expand_sets(sets, nsets, p->interp, p->spline_onchip != 0);
  std::vector<uint8_t> buf(plan_file_bytes(ps, p));
  st = encode_plan(ps, p, buf.data(), buf.size(), (uint8_t*)workspace, ws_bytes);
  if (st != IRP_OK) return st;
  // Small plans travel as kernel parameters; larger ones are copied from this
  // pageable buffer (cudaMemcpyAsync then returns after staging the data).
  return run_plan(buf.data(), (uint8_t*)workspace, ws_bytes, (cudaStream_t)stream,
                  !plan_fits_inline(buf.data()));
}

irp_status irp_reduce_set_host(const irp_set* sets, int nsets, const irp_host_io* io,
                               const irp_reduce_params* p, void* workspace, size_t ws_bytes,
                               void* stream) {
  irp_status st = check_params(sets, nsets, p);
  if (st != IRP_OK) return st;
  if (!io) return IRP_ERR_INVALID_ARG;
  for (int i = 0; i < nsets; ++i) {
    const irp_set& s = sets[i];
    const irp_host_io& h = io[i];
    if (!h.frames || h.pitch < s.W) return IRP_ERR_INVALID_ARG;
    for (int k = 0; k < s.n; ++k)
      if (!h.frames[k]) return IRP_ERR_INVALID_ARG;
    if ((h.mean && !s.mean_out) || (h.median && !s.median_out) || (h.nkept && !s.nkept_out))
      return IRP_ERR_INVALID_ARG;
    if ((h.mean || h.median || h.nkept) && h.out_pitch < s.W) return IRP_ERR_INVALID_ARG;
    if (irp_workspace_size(&s, 1, p) > ws_bytes) return IRP_ERR_WORKSPACE;
  }
  if (!workspace || !aligned(workspace, kAlign)) return IRP_ERR_WORKSPACE;
  HostPipe* hp = nullptr;
  cudaError_t e = host_pipe(&hp);
  if (e != cudaSuccess) return note_cuda(e);
  std::lock_guard<std::mutex> lock(hp->mu);  // the pipe's streams and events
  e = host_pipe_events(hp, 2 * nsets + 1);
  if (e != cudaSuccess) return note_cuda(e);
  cudaStream_t s0 = (cudaStream_t)stream;
  cudaEvent_t* ev = hp->ev.data();
  // fork: both copy streams start after the work already on the caller's stream
  e = cudaEventRecord(ev[0], s0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(hp->up, ev[0], 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(hp->down, ev[0], 0);
  for (int i = 0; i < nsets && e == cudaSuccess; ++i) {
    const irp_set& s = sets[i];
    const irp_host_io& h = io[i];
    if (h.pitch == s.W && s.raw_pitch == s.W) {
      // dense frames: one copy per run of frames contiguous on both sides
      const size_t fb = (size_t)s.W * s.H * 2;
      for (int k0 = 0; k0 < s.n && e == cudaSuccess;) {
        const uint8_t* hs = (const uint8_t*)h.frames[k0];
        const uint8_t* ds = (const uint8_t*)s.frames[k0];
        int k1 = k0 + 1;
        while (k1 < s.n && (const uint8_t*)h.frames[k1] == hs + (size_t)(k1 - k0) * fb &&
               (const uint8_t*)s.frames[k1] == ds + (size_t)(k1 - k0) * fb)
          ++k1;
        e = cudaMemcpyAsync((void*)ds, hs, (size_t)(k1 - k0) * fb, cudaMemcpyHostToDevice,
                            hp->up);
        k0 = k1;
      }
    } else {
      for (int k = 0; k < s.n && e == cudaSuccess; ++k)
        e = cudaMemcpy2DAsync((void*)s.frames[k], (size_t)s.raw_pitch * 2, h.frames[k],
                              (size_t)h.pitch * 2, (size_t)s.W * 2, (size_t)s.H,
                              cudaMemcpyHostToDevice, hp->up);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[1 + 2 * i], hp->up);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s0, ev[1 + 2 * i], 0);
    if (e != cudaSuccess) break;
    st = irp_reduce_set(&s, 1, p, workspace, ws_bytes, stream);
    if (st != IRP_OK) return st;
    e = cudaEventRecord(ev[2 + 2 * i], s0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hp->down, ev[2 + 2 * i], 0);
    auto down = [&](void* dst, const void* src, size_t es) {
      if (e != cudaSuccess || !dst) return;
      if (h.out_pitch == s.W && s.out_pitch == s.W)  // dense: one plain copy
        e = cudaMemcpyAsync(dst, src, (size_t)s.W * s.H * es, cudaMemcpyDeviceToHost, hp->down);
      else
        e = cudaMemcpy2DAsync(dst, (size_t)h.out_pitch * es, src, (size_t)s.out_pitch * es,
                              (size_t)s.W * es, (size_t)s.H, cudaMemcpyDeviceToHost, hp->down);
    };
    down(h.mean, s.mean_out, sizeof(float));
    down(h.median, s.median_out, sizeof(float));
    down(h.nkept, s.nkept_out, sizeof(uint16_t));
  }
  // join: the caller's stream continues after the last download
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], hp->down);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s0, ev[0], 0);
  return cuda_status(e);
}

irp_status irp_sync_status(void* workspace, void* stream) {
  if (!workspace || !aligned(workspace, kAlign)) return IRP_ERR_WORKSPACE;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return note_cuda(e);
  uint32_t status = 0;
  e = cudaMemcpy(&status, workspace, sizeof(uint32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return note_cuda(e);
  if (status != 0) {
    e = cudaMemset(workspace, 0, sizeof(uint32_t));
    if (e != cudaSuccess) return note_cuda(e);
  }
  return (irp_status)status;
}

// ------------------------------------------------------------------ calibrate
size_t irp_calibrate_workspace_size(int n) {
  if (n < 1) return 0;
  return sizeof(WsHeader) + align_up((size_t)(n + 1) * sizeof(FrameStats), kAlign);
}

irp_status irp_calibrate(const uint16_t* raw, int64_t raw_pitch, int64_t raw_frame_stride,
                         int W, int H, int n, const float* bias, const float* dark_rate,
                         const float* flat, int64_t master_pitch, const float* exptime_host,
                         int normalize_flat, void* out, int64_t out_pitch,
                         int64_t out_frame_stride, irp_stack_dtype dt, float* scale_out,
                         float* offset_out, void* workspace, size_t ws_bytes, void* stream) {
  if (!raw || !bias || !dark_rate || !flat || !exptime_host || !out) return IRP_ERR_INVALID_ARG;
  if (W < 1 || H < 1 || n < 1 || raw_pitch < W || master_pitch < W || out_pitch < W)
    return IRP_ERR_INVALID_ARG;
  if (raw_frame_stride < raw_pitch * H && n > 1) return IRP_ERR_INVALID_ARG;
  if (out_frame_stride < out_pitch * H && n > 1) return IRP_ERR_INVALID_ARG;
  if (dt != IRP_F32 && dt != IRP_F16_SCALED) return IRP_ERR_INVALID_ARG;
  if (dt == IRP_F16_SCALED && (!scale_out || !offset_out)) return IRP_ERR_INVALID_ARG;
  if (!aligned(raw, 2) || !aligned(bias, 4) || !aligned(dark_rate, 4) || !aligned(flat, 4) ||
      !aligned(out, dt == IRP_F32 ? 4 : 2) || !aligned(scale_out, 4) || !aligned(offset_out, 4))
    return IRP_ERR_ALIGNMENT;
  for (int k = 0; k < n; ++k)
    if (!std::isfinite(exptime_host[k])) return IRP_ERR_INVALID_ARG;
  if (!workspace || !aligned(workspace, kAlign)) return IRP_ERR_WORKSPACE;
  if (ws_bytes < irp_calibrate_workspace_size(n)) return IRP_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  WsHeader* wsh = (WsHeader*)workspace;
  FrameStats* st = (FrameStats*)((uint8_t*)workspace + sizeof(WsHeader));
  FrameStats* flat_st = st + n;
  TraceScope tr(IRP_KERNEL_CALIBRATE, s);
  cudaError_t e = launch_stats_init(st, n + 1, s);
  if (e == cudaSuccess && normalize_flat)
    e = launch_stats_frames(flat, master_pitch, 0, W, H, 1, false, nullptr, nullptr, nullptr,
                            nullptr, nullptr, flat_st, s);
  if (e != cudaSuccess) return note_cuda(e);
  CalibArgs a;
  std::memset(&a, 0, sizeof(a));
  a.raw = raw;
  a.raw_pitch = raw_pitch;
  a.raw_frame_stride = raw_frame_stride;
  a.W = W;
  a.H = H;
  a.bias = bias;
  a.dark = dark_rate;
  a.flat = flat;
  a.master_pitch = master_pitch;
  a.flat_sum = normalize_flat ? &flat_st->sum : nullptr;
  a.status = &wsh->status;
  // four pixels per vector access when every row of every operand starts on it
  a.vec = (W % 4 == 0 && raw_pitch % 4 == 0 && raw_frame_stride % 4 == 0 && aligned(raw, 8) &&
           master_pitch % 4 == 0 && aligned(bias, 16) && aligned(dark_rate, 16) &&
           aligned(flat, 16) && out_pitch % 4 == 0 && out_frame_stride % 4 == 0 &&
           aligned(out, dt == IRP_F32 ? 16 : 8)) ? 1 : 0;
  // eight pixels per thread over all frames of a launch when every row of
  // every operand starts on an 8-pixel boundary (16-byte vectors)
  const size_t oes = dt == IRP_F32 ? 4 : 2;
  const bool vec8 = W % 8 == 0 && raw_pitch % 8 == 0 && raw_frame_stride % 8 == 0 &&
                    aligned(raw, 16) && master_pitch % 4 == 0 && aligned(bias, 16) &&
                    aligned(dark_rate, 16) && aligned(flat, 16) && aligned(out, 16) &&
                    (out_pitch * (int64_t)oes) % 16 == 0 && (out_frame_stride * (int64_t)oes) % 16 == 0;
  for (int k0 = 0; k0 < n; k0 += kCalibChunk) {
    const int nk = std::min(kCalibChunk, n - k0);
    a.k0 = k0;
    for (int j = 0; j < nk; ++j) a.t[j] = exptime_host[k0 + j];
    if (dt == IRP_F16_SCALED) {
      e = vec8 ? launch_f16_stats8(a, nk, st, s) : launch_stats_raw(a, nk, st, s);
      if (e != cudaSuccess) return note_cuda(e);
    }
  }
  if (dt == IRP_F16_SCALED) {
    e = launch_f16_scaling(st, n, scale_out, offset_out, s);
    if (e != cudaSuccess) return note_cuda(e);
  }
  for (int k0 = 0; k0 < n; k0 += kCalibChunk) {
    const int nk = std::min(kCalibChunk, n - k0);
    a.k0 = k0;
    for (int j = 0; j < nk; ++j) a.t[j] = exptime_host[k0 + j];
    e = vec8 ? launch_calibrate8(a, nk, dt == IRP_F16_SCALED, out, out_pitch, out_frame_stride,
                                 scale_out, offset_out, s)
             : launch_calibrate(a, nk, dt == IRP_F16_SCALED, out, out_pitch, out_frame_stride,
                                scale_out, offset_out, s);
    if (e != cudaSuccess) return note_cuda(e);
  }
  return IRP_OK;
}

irp_status irp_frame_stats(const void* frames, int64_t pitch, int64_t frame_stride, int W, int H,
                           int n, irp_stack_dtype dt, const float* scale, const float* offset,
                           double* sum_out, double* sumsq_out, int64_t* count_out, void* stream) {
  if (!frames || !sum_out || W < 1 || H < 1 || n < 1 || pitch < W) return IRP_ERR_INVALID_ARG;
  if (n > 1 && frame_stride < pitch * H) return IRP_ERR_INVALID_ARG;
  if (dt != IRP_F32 && dt != IRP_F16_SCALED) return IRP_ERR_INVALID_ARG;
  if (dt == IRP_F16_SCALED && (!scale || !offset)) return IRP_ERR_INVALID_ARG;
  if (!aligned(frames, dt == IRP_F32 ? 4 : 2) || !aligned(sum_out, 8) || !aligned(sumsq_out, 8) ||
      !aligned(count_out, 8))
    return IRP_ERR_ALIGNMENT;
  if (n > 65535) return IRP_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  TraceScope tr(IRP_KERNEL_STATS, s);
  cudaError_t e = cudaMemsetAsync(sum_out, 0, sizeof(double) * n, s);
  if (e == cudaSuccess && sumsq_out) e = cudaMemsetAsync(sumsq_out, 0, sizeof(double) * n, s);
  if (e == cudaSuccess && count_out) e = cudaMemsetAsync(count_out, 0, sizeof(int64_t) * n, s);
  if (e == cudaSuccess)
    e = launch_stats_frames(frames, pitch, frame_stride, W, H, n, dt == IRP_F16_SCALED, scale,
                            offset, sum_out, sumsq_out, (long long*)count_out, nullptr, s);
  return cuda_status(e);
}

// ---------------------------------------------------------------------- shift
size_t irp_shift_workspace_size(int W, int H, int n, irp_interp interp) {
  if (W < 1 || H < 1 || n < 1) return 0;
  if (interp != IRP_INTERP_SPLINE3) return 0;
  return (size_t)n * coef_frame_bytes(W, H);
}

irp_status irp_shift(const void* in, int64_t in_pitch, int64_t in_frame_stride, int W, int H,
                     int n, irp_stack_dtype dt, const float* scale, const float* offset,
                     const double* dx_host, const double* dy_host, irp_interp interp, void* out,
                     int64_t out_pitch, int64_t out_frame_stride, uint8_t* valid_out,
                     void* workspace, size_t ws_bytes, void* stream) {
  (void)scale;
  (void)offset;
  if (!in || !out || !dx_host || !dy_host) return IRP_ERR_INVALID_ARG;
  if (W < 1 || H < 1 || n < 1 || in_pitch < W || out_pitch < W) return IRP_ERR_INVALID_ARG;
  if (n > 1 && (in_frame_stride < in_pitch * H || out_frame_stride < out_pitch * H))
    return IRP_ERR_INVALID_ARG;
  if (dt != IRP_F32 && dt != IRP_F16_SCALED) return IRP_ERR_INVALID_ARG;
  if (interp < IRP_INTERP_NEAREST || interp > IRP_INTERP_CUBIC) return IRP_ERR_INVALID_ARG;
  const size_t es = dt == IRP_F32 ? 4 : 2;
  if (!aligned(in, es) || !aligned(out, es)) return IRP_ERR_ALIGNMENT;
  if (in == out) return IRP_ERR_INVALID_ARG;
  for (int k = 0; k < n; ++k)
    if (!std::isfinite(dx_host[k]) || !std::isfinite(dy_host[k]) || std::fabs(dx_host[k]) > 1e9 ||
        std::fabs(dy_host[k]) > 1e9)
      return IRP_ERR_INVALID_ARG;
  const size_t need = irp_shift_workspace_size(W, H, n, interp);
  if (need > 0 && (!workspace || !aligned(workspace, kAlign) || ws_bytes < need))
    return IRP_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  TraceScope tr(IRP_KERNEL_SHIFT, s);
  const int stencil = stencil_of(interp);
  const bool f16 = dt == IRP_F16_SCALED;
  ShiftArgs sa;
  std::memset(&sa, 0, sizeof(sa));
  sa.in = in;
  sa.in_pitch = in_pitch;
  sa.in_fstride = in_frame_stride;
  sa.W = W;
  sa.H = H;
  sa.out = out;
  sa.out_pitch = out_pitch;
  sa.out_fstride = out_frame_stride;
  sa.valid_out = valid_out;
  sa.coef_pitch = coef_pitch(W);
  const int vec = (aligned(out, 4 * es) && out_pitch % 4 == 0 && out_frame_stride % 4 == 0 &&
                   (!valid_out || aligned(valid_out, 4))) ? 1 : 0;
  for (int k0 = 0; k0 < n; k0 += kShiftChunk) {
    const int nk = std::min(kShiftChunk, n - k0);
    sa.k0 = k0;
    for (int j = 0; j < nk; ++j) {
      FrameDesc& F = sa.frames[j];
      std::memset(&F, 0, sizeof(F));
      fill_geometry(F, dx_host[k0 + j], dy_host[k0 + j], W, H, interp);
      F.src = (const uint8_t*)in + (size_t)(k0 + j) * in_frame_stride * es;
      F.coef = stencil == ST_BSPLINE
                   ? (float*)((uint8_t*)workspace + (size_t)(k0 + j) * coef_frame_bytes(W, H))
                   : nullptr;
    }
    cudaError_t e = cudaSuccess;
    if (stencil == ST_BSPLINE) {
      InlinePlan inl;
      std::memset(&inl, 0, sizeof(inl));
      inl.h.nsets = 1;
      inl.h.nframes = nk;
      SetDesc& S = inl.sets[0];
      S.W = W;
      S.H = H;
      S.n = nk;
      S.src_pitch = in_pitch;
      S.coef_pitch = coef_pitch(W);
      S.ptiles_x = (W + kPrefTile - 1) / kPrefTile;
      S.ptiles_y = (H + kPrefTile - 1) / kPrefTile;
      S.pframes = 4;
      inl.h.npitems = S.ptiles_x * S.ptiles_y * ((nk + S.pframes - 1) / S.pframes);
      for (int j = 0; j < nk; ++j) inl.frames[j] = sa.frames[j];
      e = launch_prefilter_frames(&inl, inl.h.npitems, f16, s);
    }
    if (e == cudaSuccess) e = launch_shift(sa, nk, stencil, f16, vec, s);
    if (e != cudaSuccess) return note_cuda(e);
  }
  return IRP_OK;
}

// -------------------------------------------------------------------- combine
irp_status irp_combine(const void* stack, int64_t pitch, int64_t frame_stride, int W, int H, int n,
                       irp_stack_dtype dt, const float* scale, const float* offset,
                       const uint8_t* valid, const irp_clip_params* clip, float* mean_out,
                       float* median_out, uint16_t* nkept_out, uint8_t* reject_out,
                       int64_t out_pitch, void* stream) {
  if (!stack || !clip || W < 1 || H < 1 || n < 1 || pitch < W || out_pitch < W)
    return IRP_ERR_INVALID_ARG;
  if (!mean_out && !median_out && !nkept_out && !reject_out) return IRP_ERR_INVALID_ARG;
  if (n > 1 && frame_stride < pitch * H) return IRP_ERR_INVALID_ARG;
  if (n > IRP_MAX_WIDE_FRAMES) return IRP_ERR_UNSUPPORTED;
  if (dt != IRP_F32 && dt != IRP_F16_SCALED) return IRP_ERR_INVALID_ARG;
  if (dt == IRP_F16_SCALED && (!scale || !offset)) return IRP_ERR_INVALID_ARG;
  if (!clip_ok(*clip)) return IRP_ERR_INVALID_ARG;
  if (!aligned(stack, dt == IRP_F32 ? 4 : 2) || !aligned(mean_out, 4) || !aligned(median_out, 4) ||
      !aligned(nkept_out, 2) || !aligned(scale, 4) || !aligned(offset, 4))
    return IRP_ERR_ALIGNMENT;
  if (H > 65535) return IRP_ERR_UNSUPPORTED;
  CombineArgs a;
  std::memset(&a, 0, sizeof(a));
  a.stack = stack;
  a.pitch = pitch;
  a.fstride = frame_stride;
  a.W = W;
  a.H = H;
  a.n = n;
  a.scale = scale;
  a.offset = offset;
  a.valid = valid;
  a.clip = ClipArgs{clip->kappa_lo, clip->kappa_hi, clip->max_iter, clip->center, clip->ddof};
  a.mean_out = mean_out;
  a.median_out = median_out;
  a.nkept_out = nkept_out;
  a.reject_out = reject_out;
  a.out_pitch = out_pitch;
  TraceScope tr(IRP_KERNEL_COMBINE, (cudaStream_t)stream);
  const bool f16 = dt == IRP_F16_SCALED;
  return cuda_status(n > IRP_MAX_FRAMES ? launch_combine_wide(a, f16, (cudaStream_t)stream)
                                        : launch_combine(a, f16, (cudaStream_t)stream));
}

}  // extern "C"

// ---------------------------------------------------------------------------
// irp_reduce_set_noalloc: the fused reduction with its scratch in a static
// device array instead of a caller-provided workspace (see include/irp.h).
// ---------------------------------------------------------------------------

namespace {

// The scratch.  In host code this name is only a stand-in for the symbol;
// the device address is obtained per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[IRP_NOALLOC_SCRATCH_BYTES];

constexpr int kNoallocMaxDevices = 64;
constexpr size_t kNoallocPlanBytes = 64 * 1024;  // fixed host plan buffer (no heap)

// Device address of the scratch on the current device; looked up once per
// device with that device current.
cudaError_t noalloc_scratch(uint8_t** out) {
  static std::mutex mu;
  static uint8_t* addr[kNoallocMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoallocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    addr[dev] = (uint8_t*)p;
  }
  *out = addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" irp_status irp_reduce_set_noalloc(const irp_set* sets, int nsets,
                                             const irp_reduce_params* p, uint32_t* status_out,
                                             void* stream) {
  irp_status st = check_params(sets, nsets, p);
  if (st != IRP_OK) return st;
  if (!aligned(status_out, 4)) return IRP_ERR_ALIGNMENT;
  const PlanSets ps = expand_sets(sets, nsets, p->interp, p->spline_onchip != 0);
  std::vector<std::vector<int>> groups;
  group_sets(ps, p->interp, groups);
  const size_t need = make_layout(ps, p, groups).total;
  const size_t plan_bytes = plan_file_bytes(ps, p);
  if (need > IRP_NOALLOC_SCRATCH_BYTES || plan_bytes > kNoallocPlanBytes) return IRP_ERR_WORKSPACE;
  uint8_t* ws = nullptr;
  cudaError_t e = noalloc_scratch(&ws);
  if (e != cudaSuccess) return note_cuda(e);
  alignas(64) uint8_t buf[kNoallocPlanBytes];  // on the stack: no allocation
  st = encode_plan(ps, p, buf, plan_bytes, ws, IRP_NOALLOC_SCRATCH_BYTES);
  if (st != IRP_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const bool upload = !plan_fits_inline(buf);
  if (upload) {
    // the plan would be copied from `buf`, which lives on this call's stack:
    // a copy recorded into a graph would read it after the call has returned
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return note_cuda(e);
    if (cs != cudaStreamCaptureStatusNone) return IRP_ERR_UNSUPPORTED;
  }
  // the status word and work counters must start at zero for every call
  e = cudaMemsetAsync(ws, 0, sizeof(WsHeader), s);
  if (e != cudaSuccess) return note_cuda(e);
  st = run_plan(buf, ws, IRP_NOALLOC_SCRATCH_BYTES, s, upload);
  if (st != IRP_OK) return st;
  if (status_out) {
    e = cudaMemcpyAsync(status_out, ws, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return note_cuda(e);
  }
  return IRP_OK;
}

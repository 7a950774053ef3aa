#!/usr/bin/env python
"""Throughput benchmark of the fused image reduction (one JSON line on rank 0).

A step is one pass of the whole path -- calibration, alignment, sigma-clipped
mean and median -- over one batch of synthetic frames resident in HBM.

Default (``--workload headline``): the metric's own configuration.  The line's
value is the batched form: 64 frame sets of uneven shape (3 to 40 frames of
512^2 to 4096^2 uint16, bilinear, 3-sigma clip with 3 passes plus the median)
reduced by autotuned persistent launches replayed from a CUDA graph, beside
the same sets reduced by 64 plain per-set launches (``plain_mpix_s``,
``batched_over_plain``).  Sub-records: the largest plain set (32 frames of
4096^2, its HBM roofline fraction and its FP16/FP32 stack forms with errors
against the FP64 oracle), the three 10-frame bands of 1024^2 with the cubic
spline, and the served form (16-chip exposures at Poisson arrivals, p50/p99
latency).  The metric is reduced raw megapixels per second (sum of n*W*H over
a step's sets); each step is timed with CUDA events on the launch stream, L2
flushed (a 256 MB write, then a 256 MB read of a second buffer) before every
step whose data fit in L2.

--impl reference times the FP64 CPU oracle on the same workload (a bounded
sample per step) on this machine's cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    "bands": dict(desc="3 bands x 10 frames of 1024x1024 uint16, offsets +-10 px, cubic-spline "
                       "shift, 3-sigma clipped mean (3 passes) + median, the three bands in one call",
                  sets=[(1024, 1024, 10)] * 3, offset=10.0, interp="spline3", persistent=False,
                  seed=11486001),
    "bands_onchip": dict(desc="the bands workload with spline_onchip: the row pass, then one "
                              "tile kernel solving the columns and combining on chip, the "
                              "row-pass frames kept in L2",
                         sets=[(1024, 1024, 10)] * 3, offset=10.0, interp="spline3",
                         persistent=False, seed=11486001, onchip=True),
    "small": dict(desc="5 frames of 512x512 uint16, offsets +-5 px, bilinear shift, 3-sigma "
                       "clipped mean (3 passes) + median",
                  sets=[(512, 512, 5)], offset=5.0, interp="bilinear", persistent=False,
                  seed=11486000),
    "deep": dict(desc="32 frames of 4096x4096 uint16, offsets +-5 px, bilinear shift, fused FP32 "
                      "on-chip stack, 3-sigma clipped mean (3 passes) + median",
                 sets=[(4096, 4096, 32)], offset=5.0, interp="bilinear", persistent=True,
                 seed=11486002),
    "precision": dict(desc="32 frames of 4096x4096 uint16, bilinear: fused FP32 on-chip stack vs "
                           "unfused FP32 and FP16-with-per-frame-scale HBM stacks; FP64 frame sums "
                           "choose the FP16 scaling; errors against the FP64 oracle",
                      sets=[(4096, 4096, 32)], offset=5.0, interp="bilinear", persistent=True,
                      seed=11486002),
    "masked": dict(desc="32 frames of 4096x4096 uint16, offsets +-5 px, bilinear shift, a 1% "
                        "bad-pixel mask master and a saturation level of 60000 ADU (samples "
                        "touching a bad pixel leave the combine), 3-sigma clip + median",
                   sets=[(4096, 4096, 32)], offset=5.0, interp="bilinear", persistent=True,
                   seed=11486002, mask_frac=0.01, saturation=60000.0),
    "batch": dict(desc="64 frame sets, frame counts U{3..40}, sizes from {512^2, 1024^2, 2048^2, "
                       "4096^2}, bilinear: one autotuned persistent launch per frame-count bucket "
                       "replayed from a CUDA graph vs 64 plain per-set launches",
                  sets=None, offset=5.0, interp="bilinear", persistent=True, seed=11486003),
    "paper": dict(desc="the paper's timed run: 3 bands x 180 frames of 1020x1020 uint16 (n = 540), "
                       "offsets +-10 px, cubic-spline shift, 3-sigma clipped mean (3 passes) + "
                       "median; 180-frame sets: prefilter, then 8 lanes per pixel from the filtered rows",
                  sets=[(1020, 1020, 180)] * 3, offset=10.0, interp="spline3", persistent=False,
                  seed=11486005),
    "paper_band": dict(desc="one band of the paper's run: 180 frames of 1020x1020 uint16, offsets "
                            "+-10 px, cubic-spline shift, 3-sigma clipped mean (3 passes) + median",
                       sets=[(1020, 1020, 180)], offset=10.0, interp="spline3", persistent=False,
                       seed=11486005),
    "served": dict(desc="Poisson arrivals (0.5/s), each request 16 chips of 6144x6160 uint16 "
                        "reduced against a 5-frame rolling stack per chip (raw ring, resident "
                        "masters), admission by free HBM, continuous batching; p50/p99 latency "
                        "and sustained Mpix/s of new pixels",
                   sets=[(6144, 6160, 5)] * 16, offset=5.0, interp="bilinear", persistent=True,
                   seed=11486004),
}

# Scans of the paper's Sec. 3.2.2 (execution time against the frame size at
# 100 frames per band, and against the frame count at 1020 x 1020), 3 bands
# each: one JSON line with the time per point and a straight-line fit.
SWEEPS = {
    "sweep_size": dict(desc="3 bands x 100 frames of N x N uint16 (n = 300), N = 256 .. 4096, "
                            "offsets +-10 px, cubic-spline shift, 3-sigma clip + median",
                       points=[(N, N, 100) for N in (256, 512, 1020, 2048, 4096)],
                       offset=10.0, interp="spline3", persistent=False, seed=11486006),
    "sweep_frames": dict(desc="3 bands of 1020 x 1020 uint16, 10 .. 333 frames per band (n = 30 "
                              ".. 999), offsets +-10 px, cubic-spline shift, 3-sigma clip + median",
                         points=[(1020, 1020, nb) for nb in (10, 30, 60, 100, 180, 333)],
                         offset=10.0, interp="spline3", persistent=False, seed=11486007),
}

CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="irp_clocks_", suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(gpu_index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_init():
    """One rank per GPU from the torchrun environment.  The collectives run
    over NCCL; IRP_DIST_BACKEND=gloo runs them on the CPU instead (tests)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(os.environ.get("IRP_DIST_BACKEND", "nccl"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce_over_ranks(x, world, op):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch.distributed as dist
    return _reduce_over_ranks(x, world, dist.ReduceOp.MAX)


def sum_over_ranks(x, world):
    if world == 1:
        return x
    import torch.distributed as dist
    return _reduce_over_ranks(x, world, dist.ReduceOp.SUM)


def workload_shapes(workload):
    """(W, H, n) of every set of one step (of a scan: every point's 3 bands)."""
    if workload in SWEEPS:
        return [p for p in SWEEPS[workload]["points"] for _ in range(3)]
    cfg = WORKLOADS[workload]
    if cfg["sets"] is not None:
        return list(cfg["sets"])
    from paper_2008_11486_gb300 import synth
    return [(W, H, n) for (n, W, H) in synth.batch_shapes(cfg["seed"])]


def cpu_baseline(workload, steps, warmup, nthreads, as_reference=False, best=False):
    """Times the oracle as it stands on a bounded sample: one set of the
    workload (the one with the most frames), cropped to at most 256 rows and
    2048 columns, per step; the mean time per sample, or the best with
    ``best``."""
    import oracle
    from paper_2008_11486_gb300 import synth
    cfg = WORKLOADS[workload] if workload in WORKLOADS else SWEEPS[workload]
    W, H, n = max(workload_shapes(workload), key=lambda t: t[2])
    Hs, Ws = min(H, 256), min(W, 2048)
    fs = synth.make_set(Ws, Hs, n, cfg["offset"], cfg["seed"],
                        n_stars=max(1, 200 * Hs * Ws // (H * W)))
    oracle.build()
    kw = {}
    if cfg.get("mask_frac"):
        rng = np.random.default_rng(cfg["seed"])
        kw = dict(mask=(rng.random((Hs, Ws)) < cfg["mask_frac"]).astype(np.uint8),
                  saturation=cfg["saturation"])
    times = []
    for i in range(warmup + steps):
        t0 = time.perf_counter()
        oracle.reduce_set(fs, interp=cfg["interp"], nthreads=nthreads, **kw)
        dt = time.perf_counter() - t0
        if i >= warmup:
            times.append(dt)
    px = n * Ws * Hs
    mean_t = float(np.min(times) if best else np.mean(times))
    return dict(value=px / mean_t / 1e6, unit="Mpix/s", cores=nthreads, kind="oracle",
                sample=f"{n} frames of {Ws}x{Hs} (one set of the workload cropped), "
                       f"{cfg['interp']}, FP64, OpenMP {nthreads} threads",
                seconds_per_sample=mean_t)


def run_reference(args, world, rank):
    if rank != 0:
        return
    nthreads = os.cpu_count() or 1
    workload = "batch" if args.workload == "headline" else args.workload
    steps = args.steps if args.steps is not None else 3
    cb = cpu_baseline(workload, steps, args.warmup, nthreads, as_reference=True)
    cfg = WORKLOADS[workload] if workload in WORKLOADS else SWEEPS[workload]
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"],
            "unit": "Mpix/s", "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
            "ms_per_step": cb["seconds_per_sample"] * 1e3, "higher_is_better": True,
            "scaling": "strong" if workload == "batch" else "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload, "desc": cfg["desc"]},
            "cpu_baseline": {"value": cb["value"], "unit": "Mpix/s", "cores": cb["cores"],
                             "kind": "oracle", "sample": cb["sample"],
                             "cpu_model": cpu_model()},
            "e2e": {"value": cb["value"], "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def make_device_sets(shapes, cfg, dev, rank):
    import torch
    from paper_2008_11486_gb300 import core, synth
    sets = []
    for i, (W, H, n) in enumerate(shapes):
        d = synth.make_set_torch(W, H, n, cfg["offset"], cfg["seed"] + 7919 * i + 104729 * rank,
                                 dev)
        s = core.DeviceSet(frames=[d["raw"][k] for k in range(n)], bias=d["bias"],
                           dark=d["dark"], flat=d["flat"], exptime=d["exptime"], dx=d["dx"],
                           dy=d["dy"])
        s.alloc_outputs(want_nkept=False)
        s._keep.append(d["raw"])
        if cfg.get("mask_frac"):
            g = torch.Generator(device=dev)
            g.manual_seed(cfg["seed"] + 17 * i + 104729 * rank)
            s.mask = (torch.rand((H, W), generator=g, device=dev) < cfg["mask_frac"]).to(
                torch.uint8)
            s.saturation = cfg["saturation"]
        sets.append(s)
    return sets


class L2Flush:
    """Run between timed steps: a 256 MB write (twice the 129 MB L2), then a
    256 MB read of a second buffer.  The step then finds none of its data in
    L2, and no dirty line of the write is left for its kernels to write back
    (the read leaves L2 holding clean lines only)."""

    def __init__(self, dev):
        import torch
        n = 256 * 1024 * 1024 // 4
        self.w = torch.empty(n, dtype=torch.float32, device=dev)
        self.r = torch.zeros(n, dtype=torch.float32, device=dev)

    def __call__(self, i):
        self.w.fill_(float(i))
        self.r.sum()


def timed_steps(step, steps, warmup, stream, flush, world, local):
    """W untimed steps, then K steps each bracketed by CUDA events on the launch
    stream (L2 flushed before each), with launch tracing and clock sampling."""
    import torch
    from paper_2008_11486_gb300 import core
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    barrier(world)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    core.profile_enable(True)
    core.profile_read()
    wall0 = time.perf_counter()
    for i in range(steps):
        if flush is not None:
            flush(i)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier(world)
    prof = core.profile_read()
    core.profile_enable(False)
    clocks = sampler.stop()
    total_ms = max_over_ranks(float(sum(a.elapsed_time(b) for a, b in ev)), world)
    return total_ms, wall, prof, clocks


# DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum, one capture
# with --cache-control none so that L2 carries over between a step's kernels
# as in a run) of the dominant kernel kind per step, and of every kernel of
# the step, keyed by the hash of the kernel sources they were taken on:
# (source hash, dominant kind, kind bytes per step, path bytes per step).
# The captures and their commands are summarised under profiles/.
TRAFFIC = {
    # 3 bands in one call: row pass 122.39 MB, column pass 118.03 MB, the
    # vertical-tap reduction 80.01 MB
    "bands": ("ee967b6dddcc837a", "prefilter", 122_390_000 + 118_030_000, 320_420_000),
    # per band: row pass 38.38 MB, tile kernel 9.12 MB, discard 0.01 MB
    "bands_onchip": ("ee967b6dddcc837a", "reduce", 3 * 9_120_000, 3 * 47_510_000),
    "deep": ("ee967b6dddcc837a", "reduce", 1_422_410_000, 1_422_410_000),
    "precision": ("ee967b6dddcc837a", "reduce", 1_422_410_000, 1_422_410_000),
    # row pass 1131.89 MB, column pass 1519.42 MB, combine 803.59 MB
    "paper_band": ("ee967b6dddcc837a", "combine", 803_590_000, 3_454_900_000),
    # three bands of the paper_band shape: three launches of each kind
    "paper": ("ee967b6dddcc837a", "combine", 3 * 803_590_000, 3 * 3_454_900_000),
    # the 64 sets' own launches (one plain step, the first 64 of the run): the
    # batched step reduces the same tiles of the same sets, bucket by bucket
    "batch": ("ee967b6dddcc837a", "reduce", 30_563_540_000, 30_563_540_000),
}


# Warp instructions executed per step by the dominant kernel kind (ncu
# smsp__inst_executed, summed over the kind's launches in one step; the same
# captures and source hash as TRAFFIC).  Against the issue peak -- one warp
# instruction per cycle in each of an SM's 4 schedulers at the maximum SM
# clock -- they give the roofline of kernels that instruction issue, rather
# than HBM, limits.
ISSUE = {
    "bands": ("ee967b6dddcc837a", "prefilter", 21_110_000 + 22_380_000),  # rows + columns
    "bands_onchip": ("ee967b6dddcc837a", "reduce", 3 * 39_670_000),
    "deep": ("ee967b6dddcc837a", "reduce", 1_324_180_000),
    "precision": ("ee967b6dddcc837a", "reduce", 1_324_180_000),
    "paper_band": ("ee967b6dddcc837a", "combine", 1_215_470_000),
    "paper": ("ee967b6dddcc837a", "combine", 3 * 1_215_470_000),
    "batch": ("ee967b6dddcc837a", "reduce", 29_005_400_000),
}


def issue_roofline(workload, dom, dom_ms, sm_count, sm_max_mhz):
    """Issue-rate roofline of the dominant kernel kind, or None without an ncu
    instruction count for the current sources."""
    rec = ISSUE.get(workload)
    if not rec or rec[1] != dom or rec[0] != kernel_source_hash() or dom_ms <= 0:
        return None
    if sm_count < 2:  # the device's SM count could not be read
        return None
    peak = sm_count * 4 * sm_max_mhz * 1e6 / 1e9  # G warp instructions / s
    achieved = rec[2] / (dom_ms * 1e-3) / 1e9
    return {"bound": "issue", "achieved": round(achieved, 1), "peak": round(peak, 1),
            "unit": "G warp instructions/s", "frac": round(achieved / peak, 4),
            "warp_instructions": rec[2],
            "peak_basis": f"{sm_count} SMs x 4 schedulers x 1 warp instruction/cycle at "
                          f"{sm_max_mhz:.0f} MHz"}


def sm_max_mhz():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"])
    except Exception:
        return 2070.0  # GB300 maximum SM clock


def kernel_source_hash():
    import hashlib
    d = os.path.join(ROOT, "paper_2008_11486_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(d, name), "rb") as f:
                h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def path_bytes(shapes, want_nkept=False):
    """Bytes the fused path must move per step, the scope table's figure: per
    set n*P*2 (raw frames, read once) + P*12 (bias, dark, flat) + P*8 (mean,
    median), i.e. P (2n + 20).  Intermediate data a kernel writes and reads
    back (spline coefficients, a stack) are overhead, not algorithmic bytes."""
    return sum(W * H * (2 * n + 20 + (2 if want_nkept else 0)) for (W, H, n) in shapes)


def roofline(prof, steps, path_bytes_per_step, ms_per_step, workload=None, sm_count=None):
    """HBM roofline of the dominant kernel kind: the path's algorithmic bytes
    per step over that kind's device time per step (summed over its launches
    in a step).  ``path_frac`` divides the same bytes by the whole step."""
    kinds = {k: v for k, v in prof.items() if v[1] > 0}
    dom = max(kinds, key=lambda k: kinds[k][0])
    dom_ms = kinds[dom][0] / steps
    peak, peak_src = measured_peaks()
    achieved = path_bytes_per_step / (dom_ms * 1e-3) / 1e9
    traffic = None
    path_traffic = None
    rec = TRAFFIC.get(workload)
    if rec and rec[1] == dom and rec[2] is not None and rec[0] == kernel_source_hash():
        traffic = rec[2]
        path_traffic = rec[3] if len(rec) > 3 else None
    return {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
            "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
            "path_traffic": path_traffic,
            "algorithmic_bytes": path_bytes_per_step,
            "bytes_basis": "P (2n + 20) per set: raw once, masters once, mean and median once",
            "peak_source": peak_src,
            "launches_per_step": round(kinds[dom][1] / steps, 3),
            "kernel_ms": {k: round(v[0] / steps, 5) for k, v in kinds.items()},
            "path_frac": round(path_bytes_per_step / (ms_per_step * 1e-3) / 1e9 / peak, 4),
            "issue": (issue_roofline(workload, dom, dom_ms, sm_count, sm_max_mhz())
                      if sm_count else None)}


def e2e_run(sets, params, ws, e2e_steps, stream, world, warmup=3):
    """Same metric through the public host-buffer entry point
    (irp_reduce_set_host): every step copies its raw frames in from pinned
    host memory and its mean/median out, inside the timed region; each set's
    copies overlap its neighbours' reduction."""
    import torch
    from paper_2008_11486_gb300 import core
    host_raw = [torch.empty((s.n, s.H, s.W), dtype=torch.uint16, pin_memory=True) for s in sets]
    for h, s in zip(host_raw, sets):
        h.copy_(s._keep[0])
    host_out = [(torch.empty((s.H, s.W), dtype=torch.float32, pin_memory=True),
                 torch.empty((s.H, s.W), dtype=torch.float32, pin_memory=True)) for s in sets]

    def e2e_step():
        core.reduce_sets_host(sets, host_raw, host_out, params, ws=ws, stream=stream)

    for _ in range(warmup):  # the host buffers' first transfers are not timed
        e2e_step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    assert core.sync_status(ws) == 0
    ms = max_over_ranks(e0.elapsed_time(e1), world) / e2e_steps
    px = sum(s.n * s.W * s.H for s in sets)
    return {"value": round(world * px / (ms * 1e-3) / 1e6, 1), "unit": "Mpix/s",
            "api": "irp_reduce_set_host (per set: upload, reduce, download, overlapped)",
            "h2d_bytes_per_step": sum(h.numel() * 2 for h in host_raw),
            "d2h_bytes_per_step": sum(2 * s.H * s.W * 4 for s in sets)}


def sampled_errors(fs_host, outs, interp, npix=4000, seed=5):
    """Max abs/rel error of mean and median against the FP64 oracle on sampled
    pixels whose oracle clip margin is not within 1e-3 sigma of a threshold,
    and the central 90% and 95% ranges of the relative difference
    dI = (I - I_ref) / I_ref of the mean, the statistic the paper reports for
    its comparisons (Sec. 3.1)."""
    import oracle
    rng = np.random.default_rng(seed)
    H, W = fs_host.H, fs_host.W
    xs, ys = rng.integers(0, W, npix), rng.integers(0, H, npix)
    ref = oracle.reduce_set(fs_host, interp=interp, pixels=(xs, ys), nthreads=os.cpu_count() or 1)
    ok = (ref["margin"] >= 1e-3) & np.isfinite(ref["mean"])
    res = {}
    for name, (mean, med) in outs.items():
        gm, gd = mean[ys, xs].astype(np.float64), med[ys, xs].astype(np.float64)
        em, ed = np.abs(gm - ref["mean"])[ok], np.abs(gd - ref["median"])[ok]
        dI = (gm[ok] - ref["mean"][ok]) / ref["mean"][ok]
        res[name] = {"mean_max_abs": float(em.max()),
                     "mean_max_rel": float((em / np.abs(ref["mean"][ok])).max()),
                     "median_max_abs": float(ed.max()),
                     "median_max_rel": float((ed / np.abs(ref["median"][ok])).max()),
                     "mean_dI_90": [float(v) for v in np.percentile(dI, [5, 95])],
                     "mean_dI_95": [float(v) for v in np.percentile(dI, [2.5, 97.5])]}
    res["pixels"] = int(ok.sum())
    return res


def choose_steps(step, stream, min_seconds, min_steps=3, max_steps=20000):
    """Steps whose timed region lasts at least ``min_seconds`` (from the time
    of three warm steps), so that the clock samples cover it."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    per = max(e0.elapsed_time(e1) / 3 * 1e-3, 1e-7)
    return int(min(max_steps, max(min_steps, np.ceil(min_seconds / per))))


def cpu_model():
    """The host CPU's model name (x86 'model name', Arm 'CPU part' via lscpu)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "hardware")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline_both(workload):
    """The oracle on one bounded sample of the workload, single-threaded and
    on every host core, best of 3 each."""
    nproc = os.cpu_count() or 1
    one = cpu_baseline(workload, 3, 1, 1, best=True)
    allc = cpu_baseline(workload, 3, 1, nproc, best=True)
    return {"value": round(allc["value"], 3), "unit": "Mpix/s", "cores": nproc,
            "kind": "oracle", "sample": allc["sample"].rsplit(",", 1)[0],
            "timing": "best of 3 runs (after 1 warm-up) per thread count",
            "single_thread": {"value": round(one["value"], 3), "cores": 1},
            "all_cores": {"value": round(allc["value"], 3), "cores": nproc},
            "cpu_model": cpu_model(), "nproc": nproc}


def run_workload(args, name, dev, stream, world, rank, local, steps=None, min_seconds=1.0,
                 with_cpu=True, with_e2e=True):
    """Times one workload; returns its JSON record (rank 0) or None."""
    import torch
    from paper_2008_11486_gb300 import core, shard
    cfg = WORKLOADS[name]
    interp = cfg["interp"]
    heavy = name in HEAVY
    flush = None if heavy else L2Flush(dev)
    extra = {}
    shapes = workload_shapes(name)
    if name == "batch":  # sets are independent: disjoint shards per rank
        costs = [shard.set_cost(n, W, H) for (W, H, n) in shapes]
        shapes = [shapes[i] for i in shard.rank_shard(costs, world, rank)]
        scaling = "strong"
    else:
        scaling = "weak"
    sets = make_device_sets(shapes, cfg, dev, rank)
    # the batch's plain form: one non-persistent launch per set; the other
    # workloads launch as their config says (persistent CTAs pulling tiles
    # from an atomic counter measured 3% faster on 32 x 4096^2)
    persistent = bool(cfg["persistent"]) and name != "batch"
    params = core.reduce_params(interp, core.clip_params(3.0, 3), persistent=persistent,
                                spline_onchip=cfg.get("onchip", False))
    ws = core.workspace(max([core.workspace_size([s], params) for s in sets] +
                            [core.workspace_size(sets, params)]), dev)

    def plain_step():  # one call per set
        for s in sets:
            core.reduce_sets([s], params, ws=ws)

    def joint_step():  # all of the step's sets in one call
        core.reduce_sets(sets, params, ws=ws)

    step = plain_step if name == "batch" else joint_step
    if name == "batch":
        from paper_2008_11486_gb300 import batch
        for _ in range(args.warmup):
            plain_step()
        psteps = choose_steps(plain_step, stream, min_seconds)
        t_plain, _, _, pclocks = timed_steps(plain_step, psteps, 1, stream, None, world, local)
        plain_ms = t_plain / psteps
        tuner = batch.Autotuner(os.path.join(tempfile.gettempdir(), "irp_autotune.json"), reps=2)
        bparams, bcfg = tuner.params_for(sets, interp)
        br = batch.BatchReducer(sets, bparams, stream=stream)
        step = br.run
        extra["batch_status"] = br
        extra["plain"] = {"ms_per_step": round(plain_ms, 4), "steps": psteps,
                          "launches": "one irp_reduce_set call per set", "clocks": pclocks}
        extra["autotuned"] = bcfg
    if name == "precision":
        extra["unfused"] = run_unfused(sets, interp, stream, world, local)
    if name in ("paper", "paper_band"):
        # the paper's own GPU timing of the same run shape (Sec. 3.2.1, table
        # "Breakdown of t", n = 540 on one TITAN X Pascal); context only
        extra["paper_context"] = {"gpu": "TITAN X (Pascal)", "alignment_s": 0.48,
                                  "combining_s": 0.14, "bias_dark_flat_s": 1.0e-3}
    for _ in range(args.warmup):
        step()
    if steps is None:
        steps = choose_steps(step, stream, min_seconds)
    total_ms, wall, prof, clocks = timed_steps(step, steps, args.warmup, stream, flush, world,
                                               local)
    assert core.sync_status(ws) == 0
    if "batch_status" in extra:
        br = extra.pop("batch_status")
        assert br.status() == 0
        # graph replays are not traced: time the same plan's kernels in plain launches
        core.profile_enable(True)
        core.profile_read()
        for _ in range(3):
            br.plan.launch(stream)
        torch.cuda.synchronize()
        p3 = core.profile_read()
        core.profile_enable(False)
        prof = {k: (v[0] / 3 * steps, v[1] // 3 * steps) for k, v in p3.items()}
        extra["kernel_timing"] = "plain launches of the batch plan (graph replays are not traced)"
    ms_per_step = total_ms / steps
    px_local = sum(n * W * H for (W, H, n) in shapes)
    value = (world if scaling == "weak" else 1) * px_local * steps / (total_ms * 1e-3) / 1e6
    if scaling == "strong" and world > 1:
        value = sum_over_ranks(float(px_local), world) * steps / (total_ms * 1e-3) / 1e6
    if name == "batch":
        pl = extra["plain"]
        pl["mpix_s"] = round(px_local / (pl["ms_per_step"] * 1e-3) / 1e6, 1)
        extra["plain_mpix_s"] = pl["mpix_s"]
        extra["batched_over_plain"] = round(pl["ms_per_step"] / ms_per_step, 3)
    rf = roofline(prof, steps, path_bytes(shapes), ms_per_step, name,
                  sm_count=core.lib().irp_device_sm_count())
    gpu_launches = int(sum(v[1] for v in prof.values()))
    e2e = e2e_run(sets, params, ws, args.e2e_steps or (5 if heavy else 50), stream,
                  world) if with_e2e else None

    if name == "precision" and rank == 0:
        fs_host = host_frameset(sets[0])
        outs = {"fused_f32": (sets[0].mean.cpu().numpy(), sets[0].median.cpu().numpy())}
        outs.update(extra["unfused"].pop("outputs"))
        extra["errors_vs_oracle"] = sampled_errors(fs_host, outs, interp)

    cpu = None
    if rank == 0 and world == 1 and with_cpu and not args.no_cpu_baseline:
        cpu = cpu_baseline_both(name)
    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 1), "unit": "Mpix/s",
                "n_gpus": world, "steps": steps, "warmup": args.warmup,
                "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
                "scaling": scaling, "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded device generator, paper-shaped frames)",
                "config": {"workload": name, "desc": cfg["desc"],
                           "sets_per_step": len(shapes),
                           "frames_per_step": sum(n for (_, _, n) in shapes),
                           "raw_mpix_per_step": px_local / 1e6,
                           "launch": ("autotuned persistent, CUDA graph" if name == "batch" else
                                      "persistent" if persistent else "plain"),
                           "l2": ("inputs larger than L2" if heavy else
                                  "flushed before every timed step: a 256 MB write, then a 256 MB read of a second buffer"),
                           "parallelism": (f"replicas x{world} (sets independent per GPU)"
                                           if scaling == "weak" else
                                           f"disjoint set shards x{world}")},
                "roofline": rf, "e2e": e2e, "gpu_launches": gpu_launches,
                "wall_s": round(wall, 3), "clocks": clocks, "cpu_baseline": cpu}
        if "paper_context" in extra:
            extra["paper_context"]["this_step_s"] = round(ms_per_step * 1e-3, 6)
        line.update(extra)
    del sets, ws
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return line


def _sub(line, keep=("value", "unit", "ms_per_step", "steps", "config", "roofline", "e2e",
                     "gpu_launches", "clocks")):
    """A sub-record: the workload's line without the keys of the whole run."""
    return {k: v for k, v in line.items() if k in keep or k not in (
        "metric", "n_gpus", "warmup", "higher_is_better", "scaling", "vs_baseline", "dtype",
        "data", "cpu_baseline", "wall_s")}


def run_headline(args, dev, stream, world, rank, local):
    """The metric's own configuration: the batched form (value) against its
    plain per-set launches, with the largest plain set, the spline bands, one
    band of the paper's run and the served form as sub-records."""
    import torch
    line = run_workload(args, "batch", dev, stream, world, rank, local, steps=args.steps,
                        with_cpu=False)
    subs = {}
    for name in ("precision", "bands", "bands_onchip", "paper_band"):
        sub = run_workload(args, name, dev, stream, world, rank, local, with_cpu=False,
                           with_e2e=(name == "bands"))
        if rank == 0:
            subs["deep" if name == "precision" else name] = _sub(sub)
        torch.cuda.empty_cache()
    served = run_served(args, WORKLOADS["served"], dev, world, rank, local)
    torch.cuda.empty_cache()
    if rank == 0:
        subs["served"] = _sub(served, keep=("value", "unit", "ms_per_step", "steps", "config",
                                            "latency_s", "saturation", "batches", "e2e",
                                            "clocks", "admission"))
        line["subrecords"] = subs
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_both("batch")
        line["config"]["workload"] = ("batch: " + line["config"]["workload"] + " (value); "
                                      "subrecords deep, bands, bands_onchip, paper_band, "
                                      "served")
    return line


HEAVY = ("deep", "precision", "batch", "served", "masked", "paper", "paper_band")
METRIC = ("reduced Mpix/s and HBM GB/s fraction on 1 GB300, batched vs plain; "
          "p50/p99 set latency")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=None)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="headline",
                    choices=["headline"] + sorted(WORKLOADS) + sorted(SWEEPS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--requests", type=int, default=12, help="served: requests at the nominal rate")
    ap.add_argument("--rate", type=float, default=0.5, help="served: Poisson arrival rate (1/s)")
    ap.add_argument("--host-frames", type=int, default=2,
                    help="served: distinct pinned host exposures per chip, cycled by the requests")
    args = ap.parse_args()
    if args.warmup is None:
        args.warmup = 3
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    from paper_2008_11486_gb300 import build as irp_build
    irp_build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)   # non-default stream: graph capture needs one
    torch.cuda.set_stream(stream)

    if args.workload == "headline":
        if args.steps is None:
            args.steps = 20  # about one second of the batched form
        line = run_headline(args, dev, stream, world, rank, local)
    elif args.workload in SWEEPS:
        if args.steps is None:
            args.steps = 10
        line = run_sweep(args, dev, stream, world, rank, local)
    elif args.workload == "served":
        line = run_served(args, WORKLOADS["served"], dev, world, rank, local)
    else:
        line = run_workload(args, args.workload, dev, stream, world, rank, local,
                            steps=args.steps)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_sweep(args, dev, stream, world, rank, local):
    """Times one call over the 3 bands of every point of a scan (inputs larger
    than L2 at all but the smallest points; L2 flushed before each step)."""
    import torch
    from paper_2008_11486_gb300 import core
    cfg = SWEEPS[args.workload]
    flush = L2Flush(dev)
    params = core.reduce_params(cfg["interp"], core.clip_params(3.0, 3), persistent=False)
    points, t_ms, px_all, clocks = [], 0.0, 0, None
    for (W, H, nb) in cfg["points"]:
        shapes = [(W, H, nb)] * 3
        sets = make_device_sets(shapes, cfg, dev, rank)
        ws = core.workspace(core.workspace_size(sets, params), dev)
        total, _, prof, clocks = timed_steps(lambda: core.reduce_sets(sets, params, ws=ws),
                                             args.steps, args.warmup, stream, flush, world, local)
        assert core.sync_status(ws) == 0
        ms = total / args.steps
        px = 3 * nb * W * H
        points.append({"W": W, "H": H, "frames_per_band": nb, "raw_mpix": px / 1e6,
                       "ms_per_step": round(ms, 4), "mpix_s": round(world * px / (ms * 1e-3) / 1e6, 1),
                       "kernel_ms": {k: round(v[0] / args.steps, 4) for k, v in prof.items() if v[1]}})
        t_ms += ms
        px_all += px
        del sets, ws
        torch.cuda.empty_cache()
    # t = a + b * pixels: the largest relative residual shows how straight the scan is
    x = np.array([p["raw_mpix"] for p in points])
    y = np.array([p["ms_per_step"] for p in points])
    b, a = np.polyfit(x, y, 1)
    resid = float(np.max(np.abs(a + b * x - y) / y))
    return {"metric": "reduced Mpix/s", "value": round(world * px_all / (t_ms * 1e-3) / 1e6, 1),
            "unit": "Mpix/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(t_ms, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded device generator, paper-shaped frames)",
            "config": {"workload": args.workload, "desc": cfg["desc"],
                       "value": "all points' pixels over the sum of their step times",
                       "l2": "flushed before every timed step: a 256 MB write, then a 256 MB read of a second buffer",
                       "parallelism": f"replicas x{world} (sets independent per GPU)"},
            "points": points,
            "linear_fit": {"ms_offset": round(float(a), 4), "ms_per_mpix": round(float(b), 6),
                           "max_rel_residual": round(resid, 4)},
            "clocks": clocks}


def host_frameset(s):
    from paper_2008_11486_gb300 import synth
    return synth.FrameSet(raw=s._keep[0].cpu().numpy(), bias=s.bias.cpu().numpy(),
                          dark=s.dark.cpu().numpy(), flat=s.flat.cpu().numpy(),
                          exptime=np.asarray(s.exptime), dx=np.asarray(s.dx), dy=np.asarray(s.dy))


def run_unfused(sets, interp, stream, world, local):
    """Calibrate -> shift -> combine with the aligned stack materialised in HBM,
    as FP32 and as FP16 with per-frame scale and offset (chosen from FP64 frame
    sums); returns their step times and outputs."""
    import torch
    from paper_2008_11486_gb300 import core
    s = sets[0]
    raw = s._keep[0]
    res = {"outputs": {}}
    for dt in ("f32", "f16"):
        bufs = {}

        def step():
            cal, sc, of, bufs["ws"] = core.calibrate(raw, s.bias, s.dark, s.flat, s.exptime,
                                                     dtype=dt, out=bufs.get("cal"),
                                                     ws=bufs.get("ws"))
            bufs["cal"] = cal
            # invalid samples are NaN in the stack: no separate validity mask
            st, _, bufs["sws"] = core.shift(cal, s.dx, s.dy, interp, dtype=dt, scale=sc,
                                            offset=of, out=bufs.get("st"), want_valid=False,
                                            ws=bufs.get("sws"))
            bufs["st"] = st
            bufs["out"] = core.combine(st, dtype=dt, scale=sc, offset=of,
                                       clip=core.clip_params(3.0, 3))

        total_ms, _, prof, _ = timed_steps(step, 3, 1, stream, None, world, local)
        res[f"{dt}_ms_per_step"] = round(total_ms / 3, 4)
        res[f"{dt}_mpix_s"] = round(s.n * s.W * s.H / (total_ms / 3 * 1e-3) / 1e6, 1)
        res[f"{dt}_kernel_ms"] = {k: round(v[0] / 3, 4) for k, v in prof.items() if v[1]}
        o = bufs["out"]
        res["outputs"][f"unfused_{dt}"] = (o["mean"].cpu().numpy(), o["median"].cpu().numpy())
        del bufs
        torch.cuda.empty_cache()
    return res


def run_served(args, cfg, dev, world, rank, local):
    """Poisson arrivals of 16-chip exposures; p50/p99 latency at the nominal
    rate and sustained new-pixel throughput at saturation."""
    import torch
    from paper_2008_11486_gb300 import serve, synth
    shapes = cfg["sets"]
    W, H, depth = shapes[0]
    nchips = len(shapes)
    masters, host_frames = [], []
    nvar = args.host_frames  # distinct pinned host exposures per chip, cycled
    for c in range(nchips):
        d = synth.make_set_torch(W, H, nvar, cfg["offset"], cfg["seed"] + 131 * c + 104729 * rank,
                                 dev)
        masters.append((d["bias"], d["dark"], d["flat"]))
        host_frames.append([d["raw"][v].cpu().pin_memory() for v in range(nvar)])
        del d
    torch.cuda.empty_cache()
    rng = np.random.Generator(np.random.PCG64(cfg["seed"]))
    srv = serve.Server(masters, depth=depth, max_inflight=4, max_batch=2, interp=cfg["interp"],
                       device=dev, download=True)

    def make_requests(count, base):
        return [serve.Request(rid=base + r, frames=[host_frames[c][(base + r) % nvar]
                                                   for c in range(nchips)],
                              dx=rng.uniform(-5, 5, nchips), dy=rng.uniform(-5, 5, nchips))
                for r in range(count)]

    # fill the rings so every measured request reduces a full stack
    serve.run_poisson(srv, make_requests(depth - 1, 0), rate_hz=1e6)
    sampler = ClockSampler(local)
    reqs = make_requests(args.requests, 100)
    lat, wall = serve.run_poisson(srv, reqs, rate_hz=args.rate)
    phase = {"queued_s": [r.admitted - r.arrival for r in reqs],
             "upload_s": [r.uploaded - r.admitted for r in reqs],
             "upload_device_s": [r.upload_device_ms * 1e-3 for r in reqs],
             "prepare_s": [r.launched - r.uploaded for r in reqs],
             "device_s": [r.done - r.launched for r in reqs]}
    nominal = {"batches": srv.batches, "batch_sizes": list(srv.batch_sizes),
               "admitted_while_running": srv.admitted_while_running,
               "held_for_memory": srv.held_for_memory}
    sat_n = max(8, args.requests)
    from paper_2008_11486_gb300 import core
    core.profile_enable(True)
    core.profile_read()
    b0, a0 = srv.batches, srv.admitted_while_running
    sat_lat, sat_wall = serve.run_poisson(srv, make_requests(sat_n, 1000), rate_hz=1e6)
    prof = core.profile_read()
    core.profile_enable(False)
    clocks = sampler.stop()
    assert srv.status() == 0
    sizes = srv.batch_sizes[len(nominal["batch_sizes"]):]
    admission = {"nominal_rate": nominal,
                 "saturation": {"batches": srv.batches - b0,
                                "max_requests_per_batch": max(sizes) if sizes else 0,
                                "mean_requests_per_batch": round(float(np.mean(sizes)), 3)
                                if sizes else 0.0,
                                "admitted_while_running": srv.admitted_while_running - a0},
                 "workspace_bytes_per_request": srv._ws_bytes_per_request(),
                 "rule": "admitted while free HBM minus the request's batch workspace stays "
                         "above the reserve and an in-flight slot is free"}
    new_px = nchips * W * H
    sustained = sat_n * new_px / sat_wall / 1e6
    return {"metric": "reduced Mpix/s", "value": round(sustained * world, 1), "unit": "Mpix/s",
            "n_gpus": world, "steps": sat_n, "warmup": depth - 1,
            "ms_per_step": round(sat_wall / sat_n * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded device generator, paper-shaped frames)",
            "config": {"workload": "served", "desc": cfg["desc"], "chips": nchips,
                       "chip": [W, H], "stack_depth": depth, "rate_hz": args.rate,
                       "requests": args.requests, "host_frames_per_chip": args.host_frames,
                       "l2": "inputs larger than L2",
                       "parallelism": f"replicas x{world}"},
            "latency_s": {"p50": round(float(np.percentile(lat, 50)), 4),
                          "p99": round(float(np.percentile(lat, 99)), 4),
                          "max": round(float(lat.max()), 4), "rate_hz": args.rate,
                          "p50_phases": {k: round(float(np.percentile(v, 50)), 4)
                                         for k, v in phase.items()},
                          "p99_phases": {k: round(float(np.percentile(v, 99)), 4)
                                         for k, v in phase.items()}},
            "saturation": {"requests": sat_n, "wall_s": round(sat_wall, 3),
                           "p50_s": round(float(np.percentile(sat_lat, 50)), 4),
                           "p99_s": round(float(np.percentile(sat_lat, 99)), 4)},
            "batches": srv.batches, "admission": admission,
            "e2e": {"value": round(sustained * world, 1), "unit": "Mpix/s",
                    "api": "serve.Server: pinned raw frames in, mean images back in pinned "
                           "host memory; the value is end to end",
                    "h2d_bytes_per_step": new_px * 2, "d2h_bytes_per_step": new_px * 4},
            "gpu_launches": int(sum(v[1] for v in prof.values())), "clocks": clocks,
            "cpu_baseline": None, "roofline": None}


if __name__ == "__main__":
    main()

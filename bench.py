#!/usr/bin/env python
"""Throughput benchmark of the fused image reduction (one JSON line on rank 0).

A step is one pass of the whole path -- calibration, alignment, sigma-clipped
mean and median -- over one batch of synthetic frames resident in HBM.
Default workload: 3 bands x 10 frames of 1024x1024 uint16 with offsets of up
to +-10 px, cubic-spline alignment, 3-sigma clipping with 3 passes plus the
median, one set per launch.  The metric is reduced raw megapixels per second
(sum of n*W*H over the step's sets).  L2 is flushed (256 MB write) before
every timed step; each step is timed with CUDA events on the launch stream.

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
                       "shift, 3-sigma clipped mean (3 passes) + median, one set per launch",
                  sets=[(1024, 1024, 10)] * 3, offset=10.0, interp="spline3", persistent=False,
                  seed=11486001),
    "small": dict(desc="5 frames of 512x512 uint16, offsets +-5 px, bilinear shift, 3-sigma "
                       "clipped mean (3 passes) + median",
                  sets=[(512, 512, 5)], offset=5.0, interp="bilinear", persistent=False,
                  seed=11486000),
    "deep": dict(desc="32 frames of 4096x4096 uint16, offsets +-5 px, bilinear shift, fused FP32 "
                      "on-chip stack, 3-sigma clipped mean (3 passes) + median",
                 sets=[(4096, 4096, 32)], offset=5.0, interp="bilinear", persistent=False,
                 seed=11486002),
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
                 "-lms", "200", "-i", str(gpu_index)], stdout=self.f, stderr=subprocess.DEVNULL)
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
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def algorithmic_bytes(kind, sets, interp, want_nkept=False):
    """Bytes one launch of ``kind`` must move, per the path's data flow:
    reduce from raw: n*P*2 (raw) + P*12 (bias, dark, flat) + P*8 (mean, median)
    reduce from spline coefficients: n*P*4 + P*8
    prefilter: n*P*2 (raw) + P*12 (masters) + n*P*4 (coefficients)."""
    tot = 0
    for (W, H, n) in sets:
        P = W * H
        out = P * (8 + (2 if want_nkept else 0))
        if kind == "reduce":
            tot += (n * P * 4 + out) if interp == "spline3" else (n * P * 2 + P * 12 + out)
        elif kind == "prefilter":
            tot += n * P * 2 + P * 12 + n * P * 4
    return tot


def cpu_baseline(workload, steps, warmup, nthreads, as_reference=False):
    """Times the oracle as it stands on a bounded sample: one set of the
    workload, cropped to at most 256 rows, per step."""
    import oracle
    from paper_2008_11486_gb300 import synth
    cfg = WORKLOADS[workload]
    W, H, n = cfg["sets"][0]
    Hs = min(H, 256)
    fs = synth.make_set(W, Hs, n, cfg["offset"], cfg["seed"], n_stars=max(1, 200 * Hs // H))
    oracle.build()
    times = []
    for i in range(warmup + steps):
        t0 = time.perf_counter()
        oracle.reduce_set(fs, interp=cfg["interp"], nthreads=nthreads)
        dt = time.perf_counter() - t0
        if i >= warmup:
            times.append(dt)
    px = n * W * Hs
    mean_t = float(np.mean(times))
    return dict(value=px / mean_t / 1e6, unit="Mpix/s", cores=nthreads, kind="oracle",
                sample=f"{n} frames of {W}x{Hs} (one set of the workload cropped to {Hs} rows), "
                       f"{cfg['interp']}, FP64, OpenMP {nthreads} threads",
                seconds_per_sample=mean_t)


def run_reference(args, world, rank):
    if rank != 0:
        return
    nthreads = os.cpu_count() or 1
    cb = cpu_baseline(args.workload, args.steps, args.warmup, nthreads, as_reference=True)
    cfg = WORKLOADS[args.workload]
    line = {"impl": "reference", "metric": "reduced Mpix/s", "value": cb["value"],
            "unit": "Mpix/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": cb["seconds_per_sample"] * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": cfg["desc"]},
            "cpu_baseline": {"value": cb["value"], "unit": "Mpix/s", "cores": cb["cores"],
                             "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": cb["value"], "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bands", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=50)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    from paper_2008_11486_gb300 import build as irp_build
    from paper_2008_11486_gb300 import core, synth
    irp_build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = WORKLOADS[args.workload]
    interp = cfg["interp"]
    stream = torch.cuda.current_stream()

    # ---- inputs resident in HBM (same recipe as synth.make_set, device RNG)
    sets = []
    for i, (W, H, n) in enumerate(cfg["sets"]):
        d = synth.make_set_torch(W, H, n, cfg["offset"], cfg["seed"] + 7919 * i + 104729 * rank,
                                 dev)
        s = core.DeviceSet(frames=[d["raw"][k] for k in range(n)], bias=d["bias"],
                           dark=d["dark"], flat=d["flat"], exptime=d["exptime"], dx=d["dx"],
                           dy=d["dy"])
        s.alloc_outputs(want_nkept=False)
        s._keep.append(d["raw"])
        sets.append(s)
    params = core.reduce_params(interp, core.clip_params(3.0, 3), persistent=cfg["persistent"])
    ws_bytes = max(core.workspace_size([s], params) for s in sets)
    ws = core.workspace(ws_bytes, dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    px_per_step = sum(n * W * H for (W, H, n) in cfg["sets"])

    def step():
        for s in sets:
            core.reduce_sets([s], params, ws=ws)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert core.sync_status(ws) == 0

    # ---- timed region
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    core.profile_enable(True)
    core.profile_read()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier(world)
    prof = core.profile_read()
    core.profile_enable(False)
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(float(sum(step_ms)), world)
    assert core.sync_status(ws) == 0
    ms_per_step = total_ms / args.steps
    value = world * px_per_step * args.steps / (total_ms * 1e-3) / 1e6

    # ---- roofline of the dominant kernel (device time summed over the timed region)
    kinds = {k: v for k, v in prof.items() if v[1] > 0 and k != "stats"}
    dom = max(kinds, key=lambda k: kinds[k][0])
    dom_ms, dom_launches = kinds[dom]
    avg_launch_ms = dom_ms / dom_launches
    launches_per_step = dom_launches / args.steps
    per_launch = [s for s in cfg["sets"]]
    bytes_per_launch = algorithmic_bytes(dom, per_launch, interp) / max(launches_per_step, 1)
    peak, peak_src = measured_peaks()
    achieved = bytes_per_launch / (avg_launch_ms * 1e-3) / 1e9
    gpu_launches = int(sum(v[1] for v in prof.values()))
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                "peak_source": peak_src,
                "kernel_ms": {k: round(v[0] / args.steps, 5) for k, v in prof.items() if v[1]},
                "path_frac": round(algorithmic_bytes("reduce", per_launch, "bilinear") /
                                   (ms_per_step * 1e-3) / 1e9 / peak, 4)}

    # ---- end to end through the public API with host buffers
    host_raw = [torch.empty((s.n, s.H, s.W), dtype=torch.uint16, pin_memory=True) for s in sets]
    for h, s in zip(host_raw, sets):
        h.copy_(s._keep[0])
    host_out = [(torch.empty((s.H, s.W), dtype=torch.float32, pin_memory=True),
                 torch.empty((s.H, s.W), dtype=torch.float32, pin_memory=True)) for s in sets]
    h2d = sum(h.numel() * 2 for h in host_raw)
    d2h = sum(2 * s.H * s.W * 4 for s in sets)

    def e2e_step():
        for h, s in zip(host_raw, sets):
            s._keep[0].copy_(h, non_blocking=True)
        step()
        for (m, d), s in zip(host_out, sets):
            m.copy_(s.mean, non_blocking=True)
            d.copy_(s.median, non_blocking=True)

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.e2e_steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world) / args.e2e_steps
    e2e = {"value": round(world * px_per_step / (e2e_ms * 1e-3) / 1e6, 1), "unit": "Mpix/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(args.workload, 2, 1, os.cpu_count() or 1)
        cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        cpu["value"] = round(cpu["value"], 3)

    if rank == 0:
        line = {"metric": "reduced Mpix/s", "value": round(value, 1), "unit": "Mpix/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded device generator, paper-shaped frames)",
                "config": {"workload": args.workload, "desc": cfg["desc"],
                           "frames_per_step": sum(n for (_, _, n) in cfg["sets"]),
                           "raw_mpix_per_step": px_per_step / 1e6,
                           "l2": "flushed by a 256 MB write before every timed step",
                           "parallelism": f"replicas x{world} (sets independent per GPU)"},
                "roofline": roofline, "e2e": e2e, "gpu_launches": gpu_launches,
                "wall_s": round(wall, 3), "clocks": clocks, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Batched reduction of many frame sets of uneven shape, and its autotuner.

``BatchReducer`` encodes all sets into one plan (pinned host memory), launches
it as persistent CTAs pulling (set, tile) work items longest-first, and
captures that launch in a CUDA graph so that every later pass is one graph
replay.  ``Autotuner`` picks the work distribution (persistent CTAs pulling
tiles, or one CTA per tile), the tile height (rows per warp) and the
persistent grid size for a batch signature by timing the candidates on the
batch itself with CUDA events, and keeps the winners in a JSON cache.  The
tile width is one warp (a lane per output column) and the frames a CTA
stages at once are fixed by its shared memory, so they are not tuned.
"""
from __future__ import annotations

import json
import math
import os
import threading

import torch

from . import core
from ._binding import lib


def _bucket(n: int) -> int:
    for b in (4, 5, 6, 8, 10, 12, 16, 24, 32, 40, 48, 64):
        if n <= b:
            return b
    return 64


def _alt_rows(bucket: int, interp: str) -> int:
    """The bucket's other rows-per-warp choice (the library's default is the
    first): 4 / 2 up to 16 frames; above, 2 / 1 up to 40 frames and for the
    Keys stencil, else 1 / 2."""
    if bucket <= 16:
        return 2
    return 1 if bucket <= 40 or interp == "cubic" else 2


def signature(sets, interp: str) -> str:
    """Batch signature: interpolation, and the multiset of (frame-count bucket,
    log2 size class) of the sets."""
    keys = sorted((_bucket(s.n), int(round(math.log2(max(1, s.W * s.H))))) for s in sets)
    return f"{interp}|" + ",".join(f"{b}x{c}" for b, c in keys)


class Autotuner:
    """Times candidate launch configurations and caches the best per signature.

    Candidates: rows per warp (0 = bucket default, or the alternative height)
    and, for persistent launches, the grid as 1x / 2x / 4x the SM count
    (0 = occupancy-derived), or one CTA per tile (persistent False)."""

    def __init__(self, cache_path: str | None = None, reps: int = 3):
        self.cache_path = cache_path
        self.reps = reps
        self._lock = threading.Lock()
        self.cache = {}
        if cache_path and os.path.exists(cache_path):
            try:
                with open(cache_path) as f:
                    cache = json.load(f)
                if isinstance(cache, dict):
                    self.cache = cache
            except (OSError, ValueError):
                pass  # an unreadable cache is re-tuned, not fatal

    @staticmethod
    def candidates(sets, persistent: bool, interp: str = "bilinear"):
        sms = int(lib().irp_device_sm_count()) or 1
        rows = [0]
        alts = {_alt_rows(_bucket(s.n), interp) for s in sets}
        rows += sorted(alts)
        grids = [0, sms, 2 * sms, 4 * sms] if persistent else [0]
        cands = [dict(rows_per_warp=r, max_ctas=g, persistent=persistent)
                 for r in rows for g in grids]
        if persistent:
            cands += [dict(rows_per_warp=r, max_ctas=0, persistent=False) for r in rows]
        return cands

    def _time(self, sets, params, stream) -> float:
        plan = core.Plan(sets, params)
        for _ in range(2):
            plan.launch(stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        best = float("inf")
        for _ in range(self.reps):
            e0.record(stream)
            plan.launch(stream)
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    def tune(self, sets, interp="bilinear", clip=None, persistent=True, stream=None):
        """Returns (best config dict, {config: ms}) after timing every candidate."""
        stream = stream if stream is not None else torch.cuda.current_stream()
        results = {}
        for cand in self.candidates(sets, persistent, interp):
            p = core.reduce_params(interp, clip, **cand)
            results[json.dumps(cand, sort_keys=True)] = self._time(sets, p, stream)
        best = min(results, key=results.get)
        return json.loads(best), results

    def params_for(self, sets, interp="bilinear", clip=None, persistent=True, stream=None):
        key = signature(sets, interp) + f"|persistent={int(persistent)}"
        with self._lock:
            cfg = self.cache.get(key)
        if cfg is None:
            cfg, _ = self.tune(sets, interp, clip, persistent, stream)
            with self._lock:
                self.cache[key] = cfg
                if self.cache_path:
                    tmp = self.cache_path + ".tmp"
                    with open(tmp, "w") as f:
                        json.dump(self.cache, f, indent=1, sort_keys=True)
                    os.replace(tmp, self.cache_path)
        cfg = {"persistent": persistent, **cfg}  # caches written before the knob existed
        return core.reduce_params(interp, clip, **cfg), cfg


class BatchReducer:
    """One persistent launch over all sets, replayed from a CUDA graph."""

    def __init__(self, sets, params, stream=None, use_graph=True):
        self.sets = list(sets)
        self.params = params
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.plan = core.Plan(self.sets, params)
        self.graph = None
        if use_graph:
            torch.cuda.synchronize()
            with torch.cuda.stream(self.stream):
                self.plan.launch(self.stream)  # warm the module load and smem opt-in
            self.stream.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(self.stream):
                with torch.cuda.graph(g, stream=self.stream):
                    self.plan.launch(self.stream)
            self.graph = g

    def run(self):
        if self.graph is not None:
            with torch.cuda.stream(self.stream):
                self.graph.replay()
        else:
            self.plan.launch(self.stream)

    def status(self) -> int:
        return core.sync_status(self.plan.ws, self.stream)

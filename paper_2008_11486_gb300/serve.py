"""Continuous-batching reduction service.

A request is one exposure of a multi-chip camera: one new raw frame per chip
plus its dither offset.  Each chip keeps its calibration masters resident on
the device and a ring of its most recent raw frames; a request is reduced as
one frame set per chip made of the new frame and the ``depth - 1`` previous
ones (a rolling reference stack).

Scheduling:
  * admission: a request is admitted when an in-flight slot is free and the
    device keeps its reserve free after the request's own device bytes
    (``torch.cuda.mem_get_info``).  Frames, outputs and masters live in rings
    allocated once; what a request may still allocate is the workspace of the
    batch it joins, unless a free workspace of a completed batch is large
    enough.  A request held back for memory waits at the head of the queue
    until a batch completes.  Its outputs stay valid until ``out_slots``
    newer requests have been admitted;
    admitted requests copy their new frames into the chip rings on a copy
    stream (pinned host memory -> HBM);
  * batching: at every scheduler tick the admitted requests whose copies have
    landed are reduced together in one persistent launch (all their chip sets
    in one plan), on the compute stream, while newer requests keep uploading.
    While a batch is on the device, ready requests wait for it (up to
    ``max_batch`` of them) and then go together in the next launch: requests
    that arrive during a batch are admitted, upload behind it and join the
    next one (continuous batching);
  * completion: an event per batch; a request's latency is the time from its
    arrival to the host seeing its outputs ready;
  * errors: a request the rings cannot take (a frame of the wrong shape or
    type, a non-finite offset) completes at submission with its own status;
    each batch's device status word is cleared before its launch and
    copied back to pinned host memory behind it.  A batch that reports an
    error (a bad flat, a timed-out wait) has its requests reduced again one by
    one, so that only the failing ones carry the error in ``Request.status``
    and the others complete normally.
Each result depends only on its own frames and masters, so it is the same
alone and inside any batch.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time

import numpy as np
import torch

from . import core


CANCELLED = -1  # Request.status of a withdrawn request (not a library status)


@dataclasses.dataclass
class Request:
    rid: int
    frames: list          # per chip: pinned host uint16 [H, W]
    dx: np.ndarray        # per chip offset of the new frame
    dy: np.ndarray
    exptime: float = 60.0
    arrival: float = 0.0
    admitted: float = 0.0  # its frames' copies queued
    uploaded: float = 0.0  # the scheduler saw its copies complete
    upload_device_ms: float = 0.0  # device time of its copies (CUDA events on the copy stream)
    launched: float = 0.0  # its reduction queued
    done: float = 0.0
    outputs: list = None  # per chip (mean, median) device tensors (views of the output ring)
    host_means: list = None  # per chip pinned host mean images (servers that download)
    out_slot: int = 0
    status: int = 0       # device status of its reduction (0 = IRP_OK), set on completion
    _copy_events: tuple = dataclasses.field(default=None, repr=False)  # (start, end) of its upload


class Chip:
    """Resident masters, the raw-frame ring and the output ring of one
    detector chip (all allocated once)."""

    def __init__(self, bias, dark, flat, depth: int, slots: int, out_slots: int):
        self.bias, self.dark, self.flat = bias, dark, flat
        self.H, self.W = bias.shape
        self.depth = depth
        self.ring = torch.empty((slots, self.H, self.W), dtype=torch.uint16, device=bias.device)
        # mean and median of the last out_slots requests
        self.out = torch.empty((out_slots, 2, self.H, self.W), dtype=torch.float32,
                               device=bias.device)
        self.out_slots = out_slots
        self.slot_dx = np.zeros(slots)
        self.slot_dy = np.zeros(slots)
        self.slot_t = np.full(slots, 60.0, dtype=np.float32)
        self.count = 0        # frames written so far
        self.slots = slots

    def next_slot(self) -> int:
        return self.count % self.slots

    def stack_slots(self, upto: int):
        """Ring slots of the set ending with frame number ``upto`` (oldest first)."""
        first = max(0, upto - self.depth + 1)
        return [k % self.slots for k in range(first, upto + 1)]


class Server:
    def __init__(self, masters, depth=5, max_inflight=2, interp="bilinear", clip=None,
                 hbm_reserve_bytes=2 << 30, device="cuda", out_slots=None, download=False,
                 max_batch=None):
        self.device = torch.device(device)
        self.depth = depth
        self.max_inflight = max_inflight
        self.max_batch = max_batch if max_batch is not None else max_inflight
        self.interp = interp
        self.clip = clip
        self.reserve = hbm_reserve_bytes
        # ring slots: depth for the stack plus one per request that may still be
        # reading when the next one writes
        # output slots: a request's (mean, median) stay valid until out_slots
        # newer requests have been admitted
        self.out_slots = out_slots if out_slots is not None else max_inflight + 2
        if self.out_slots < max_inflight:
            raise ValueError("out_slots must cover the requests in flight")
        self.chips = [Chip(b, d, f, depth, depth + max_inflight, self.out_slots)
                      for (b, d, f) in masters]
        self.admitted = 0
        self.copy_stream = torch.cuda.Stream(device=self.device)
        self.compute_stream = torch.cuda.Stream(device=self.device)
        self.pending = collections.deque()   # arrived, not admitted
        self.uploading = []                  # (request, frame numbers, copy event)
        self.running = []                    # (requests, completion event, plan, ws,
                                             #  status slot, each request's sets)
        self.done = []
        self.lock = threading.Lock()
        self.ws_free = []                    # workspaces of completed batches
        self.ws_all = []
        self.batches = 0
        # one host status word per batch in flight (a batch holds at least one
        # request, so at most max_inflight batches run at once)
        self.status_host = torch.zeros(max_inflight, dtype=torch.int32,
                                       pin_memory=torch.cuda.is_available())
        self.status_free = list(range(max_inflight))
        self.failed = []                     # completed requests whose status is not OK
        self._ws_per_req = None              # workspace bytes of one request's sets
        self.held_for_memory = 0             # admissions deferred for lack of free HBM
        self.batch_sizes = []                # requests per launched batch
        self.admitted_while_running = 0      # admissions while a batch was on the device
        # download: each request's mean images are copied back to pinned host
        # memory behind its batch (Request.host_means), before it completes
        self.download = download
        self.host_out = None
        if download:
            pin = torch.cuda.is_available()
            self.host_out = [[torch.empty((c.H, c.W), dtype=torch.float32, pin_memory=pin)
                              for c in self.chips] for _ in range(self.out_slots)]

    # ---------------------------------------------------------------- intake
    def submit(self, req: Request):
        """Queues a request, or completes it at once with IRP_ERR_INVALID_ARG
        (1) in ``status`` when the rings cannot take it: the other requests
        are not affected."""
        req.arrival = time.perf_counter()
        st = self._validate(req)
        with self.lock:
            if st:
                req.status = st
                req.done = req.arrival
                self.done.append(req)
                self.failed.append(req)
            else:
                self.pending.append(req)

    def cancel(self, rid: int) -> bool:
        """Withdraws a request that has not been admitted yet: it completes at
        once with ``status = CANCELLED`` and takes no ring slot.  An admitted
        request runs to completion.  Returns whether the request was withdrawn."""
        with self.lock:
            for i, r in enumerate(self.pending):
                if r.rid == rid:
                    del self.pending[i]
                    r.status = CANCELLED
                    r.done = time.perf_counter()
                    self.done.append(r)
                    return True
        return False

    def _validate(self, req) -> int:
        """One uint16 frame of its chip's shape per chip, finite offsets and a
        finite, non-negative exposure time."""
        if len(req.frames) != len(self.chips):
            return 1
        for chip, f in zip(self.chips, req.frames):
            if not isinstance(f, torch.Tensor) or f.dtype != torch.uint16 or \
                    tuple(f.shape) != (chip.H, chip.W):
                return 1
        dx = np.asarray(req.dx, dtype=np.float64)
        dy = np.asarray(req.dy, dtype=np.float64)
        if dx.shape != (len(self.chips),) or dy.shape != dx.shape or \
                not (np.isfinite(dx).all() and np.isfinite(dy).all()):
            return 1
        if not (np.isfinite(req.exptime) and req.exptime >= 0):
            return 1
        return 0

    def _ws_bytes_per_request(self) -> int:
        """Workspace bytes of one request's chip sets (every request has the
        same shapes, so this is computed once, from the chips' first ring
        slots)."""
        if self._ws_per_req is None:
            params = core.reduce_params(self.interp, self.clip, persistent=True)
            sets = [core.DeviceSet(frames=[chip.ring[k] for k in range(self.depth)],
                                   bias=chip.bias, dark=chip.dark, flat=chip.flat,
                                   exptime=chip.slot_t[:self.depth],
                                   dx=chip.slot_dx[:self.depth], dy=chip.slot_dy[:self.depth],
                                   mean=chip.out[0, 0], median=chip.out[0, 1])
                    for chip in self.chips]
            self._ws_per_req = int(core.workspace_size(sets, params))
        return self._ws_per_req

    def _request_bytes(self, req) -> int:
        """Device bytes that admitting ``req`` may allocate.  Its frames and
        outputs go to rings allocated once, so only the workspace of the batch
        it joins counts: that batch holds it and the requests uploading now,
        and a free workspace of that size from an earlier batch is reused."""
        need = self._ws_bytes_per_request() * (len(self.uploading) + 1)
        if any(w.numel() >= need for w in self.ws_free):
            return 0
        return need

    def _inflight(self) -> int:
        return len(self.uploading) + sum(len(r[0]) for r in self.running)

    # -------------------------------------------------------------- scheduling
    def _admit(self):
        while True:
            with self.lock:
                if not self.pending or self._inflight() >= self.max_inflight:
                    return
                req = self.pending[0]
            free, _ = torch.cuda.mem_get_info(self.device)
            if free - self._request_bytes(req) < self.reserve:
                self.held_for_memory += 1
                return
            with self.lock:
                # cancel() may have withdrawn the head while the lock was free
                if not self.pending or self.pending[0] is not req:
                    continue
                self.pending.popleft()
            nums = []
            with torch.cuda.stream(self.copy_stream):
                ev0 = torch.cuda.Event(enable_timing=True)
                ev0.record(self.copy_stream)
                for c, (chip, frame) in enumerate(zip(self.chips, req.frames)):
                    slot = chip.next_slot()
                    chip.ring[slot].copy_(frame, non_blocking=True)
                    chip.slot_dx[slot] = req.dx[c]
                    chip.slot_dy[slot] = req.dy[c]
                    chip.slot_t[slot] = req.exptime
                    nums.append(chip.count)
                    chip.count += 1
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(self.copy_stream)
            req.admitted = time.perf_counter()
            req._copy_events = (ev0, ev)
            req.out_slot = self.admitted % self.out_slots
            self.admitted += 1
            if self.running:
                self.admitted_while_running += 1
            self.uploading.append((req, nums, ev))

    def _launch(self):
        ready, waiting = [], []
        now = time.perf_counter()
        for u in self.uploading:  # one query per upload, so none is lost in between
            if u[2].query():
                if not u[0].uploaded:
                    u[0].uploaded = now
                ready.append(u)
            else:
                waiting.append(u)
        if not ready:
            return
        if self.running and len(ready) < self.max_batch:
            return  # the device is busy: ready requests join the next batch
        ready = ready[:self.max_batch]
        taken = {id(u) for u in ready}
        self.uploading = [u for u in self.uploading if id(u) not in taken]
        sets, reqs, per_req = [], [], []
        for req, nums, ev in ready:
            self.compute_stream.wait_event(ev)
            req.outputs = []
            per_req.append([])
            for chip, num in zip(self.chips, nums):
                slots = chip.stack_slots(num)
                s = core.DeviceSet(frames=[chip.ring[k] for k in slots], bias=chip.bias,
                                   dark=chip.dark, flat=chip.flat, exptime=chip.slot_t[slots],
                                   dx=chip.slot_dx[slots], dy=chip.slot_dy[slots],
                                   mean=chip.out[req.out_slot, 0],
                                   median=chip.out[req.out_slot, 1])
                sets.append(s)
                per_req[-1].append(s)
                req.outputs.append((s.mean, s.median))
            reqs.append(req)
        params = core.reduce_params(self.interp, self.clip, persistent=True)
        need = core.workspace_size(sets, params)
        ws = None
        for i, w in enumerate(self.ws_free):
            if w.numel() >= need:
                ws = self.ws_free.pop(i)
                break
        if ws is None:
            with torch.cuda.stream(self.compute_stream):  # zeroed in stream order
                ws = core.workspace(need, self.device)
            self.ws_all.append(ws)
        plan = core.Plan(sets, params, device=self.device, ws=ws)  # pinned plan: no host wait
        slot = self.status_free.pop()
        with torch.cuda.stream(self.compute_stream):
            status = ws[:4].view(torch.int32)
            status.zero_()  # this batch's status word starts clear
        plan.launch(self.compute_stream)
        with torch.cuda.stream(self.compute_stream):
            self.status_host[slot:slot + 1].copy_(status, non_blocking=True)
            if self.download:
                for r in reqs:
                    r.host_means = self.host_out[r.out_slot]
                    for c, (mean, _) in enumerate(r.outputs):
                        r.host_means[c].copy_(mean, non_blocking=True)
        t = time.perf_counter()
        for r in reqs:
            r.launched = t
        done_ev = torch.cuda.Event()
        done_ev.record(self.compute_stream)
        self.running.append((reqs, done_ev, plan, ws, slot, per_req))
        self.batches += 1
        self.batch_sizes.append(len(reqs))

    def _isolate(self, reqs, per_req, ws):
        """A batch reported a device error: each of its requests is reduced
        again alone (its ring slots are still intact: it is still in flight),
        and only the failing ones keep the error.  The others' outputs are
        recomputed, with the same values."""
        params = core.reduce_params(self.interp, self.clip, persistent=True)
        core.sync_status(ws, self.compute_stream)  # clears the batch's latched status
        for req, sets in zip(reqs, per_req):
            core.reduce_sets(sets, params, ws=ws, stream=self.compute_stream)
            req.status = core.sync_status(ws, self.compute_stream)
            if req.status != 0:
                self.failed.append(req)

    def _complete(self):
        still = []
        for entry in self.running:
            reqs, ev, plan, ws, slot, per_req = entry
            if ev.query():
                st = int(self.status_host[slot])
                self.status_free.append(slot)
                if st != 0:
                    self._isolate(reqs, per_req, ws)
                t = time.perf_counter()
                for r in reqs:
                    r.done = t
                    ev0, ev1 = r._copy_events
                    r.upload_device_ms = ev0.elapsed_time(ev1)
                    r._copy_events = None
                    self.done.append(r)
                self.ws_free.append(ws)
            else:
                still.append(entry)
        self.running = still

    def tick(self):
        self._complete()
        self._admit()
        self._launch()

    def idle(self) -> bool:
        with self.lock:
            return not self.pending and not self.uploading and not self.running

    def drain(self, timeout_s=600.0):
        t0 = time.perf_counter()
        while not self.idle():
            self.tick()
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError("server did not drain")
            time.sleep(50e-6)
        self._complete()

    # ------------------------------------------------------ checkpoint / resume
    def snapshot(self) -> dict:
        """Host copy of the state a restarted server needs to continue the
        rolling stacks: each chip's raw-frame ring with its slots' offsets and
        exposure times, the frame counters and the admission count.  The
        masters are the caller's and are not copied.  Needs an idle server
        (``drain()`` first)."""
        if not self.idle():
            raise RuntimeError("snapshot needs an idle server: drain() first")
        if self.device.type == "cuda":
            torch.cuda.synchronize(self.device)
        return {"depth": self.depth, "admitted": self.admitted,
                "chips": [{"ring": c.ring.cpu().clone(), "dx": c.slot_dx.copy(),
                           "dy": c.slot_dy.copy(), "t": c.slot_t.copy(), "count": c.count}
                          for c in self.chips]}

    def restore(self, snap: dict) -> None:
        """Loads a snapshot into an idle server with the same chips, stack
        depth and ring size; the next request continues the stacks where the
        snapshot's server stopped."""
        if not self.idle():
            raise RuntimeError("restore needs an idle server")
        if snap["depth"] != self.depth or len(snap["chips"]) != len(self.chips) or any(
                tuple(s["ring"].shape) != tuple(c.ring.shape)
                for s, c in zip(snap["chips"], self.chips)):
            raise ValueError("snapshot of a server with other chips, depth or ring size")
        for c, s in zip(self.chips, snap["chips"]):
            c.ring.copy_(s["ring"])
            c.slot_dx[:] = s["dx"]
            c.slot_dy[:] = s["dy"]
            c.slot_t[:] = s["t"]
            c.count = int(s["count"])
        self.admitted = int(snap["admitted"])
        if self.device.type == "cuda":
            torch.cuda.synchronize(self.device)

    def status(self) -> int:
        """Synchronises and returns the first non-OK status of any completed
        request (withdrawn ones aside), or of any batch's workspace."""
        st = next((r.status for r in self.done if r.status not in (0, CANCELLED)), 0)
        for ws in self.ws_all:
            s = core.sync_status(ws, self.compute_stream)
            st = st or s
        return st


def run_poisson(server: Server, requests, rate_hz: float, seed: int = 11486004):
    """Submits requests at Poisson arrival times (rate_hz) while driving the
    scheduler; returns per-request latencies (s) and the wall time."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_hz, size=len(requests))
    t0 = time.perf_counter()
    due = t0 + np.cumsum(gaps)
    i = 0
    while i < len(requests) or not server.idle():
        now = time.perf_counter()
        while i < len(requests) and now >= due[i]:
            server.submit(requests[i])
            i += 1
        server.tick()
        time.sleep(20e-6)
    wall = time.perf_counter() - t0
    lat = np.array([r.done - r.arrival for r in requests])
    return lat, wall

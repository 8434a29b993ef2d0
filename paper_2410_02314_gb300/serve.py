"""Serving loop: frame stacks of mixed sizes arrive over time and are localized with
continuous batching on one GPU.

* Weights and per-size workspaces stay resident: each slot is one library context (its own
  workspace and TMA descriptors, cached per frame size) driving its own CUDA stream.
* Admission: requests wait in arrival order and start as soon as a slot is free and their
  device memory (frames + record buffer) fits the HBM budget next to the requests already
  running.  Requests that arrive while others run are admitted the moment a slot and memory
  free up, and their kernels interleave with the running ones on the device.
* Each request's records are the same alone and in the mix: every frame is computed
  independently and deterministically (no reduction depends on what else is on the GPU).
* Latency is measured from arrival to records in host memory; the report gives p50 / p99
  latency and sustained frames/s.

The paper's own inference frame (Sec. 2.2) overlaps loading and inference with processes
and preloads images into memory; here pinned host buffers and asynchronous copies on each
slot's stream play that role.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    frames: object  # host uint16 [T,H,W] (pinned torch tensor for the GPU executor)
    arrival: float  # seconds since the start of the run
    p_min: float = 0.5
    gain: float = 1.0
    offset: float = 100.0
    gain_map: object = None  # device float32 [H,W] or None
    offset_map: object = None
    admitted: float = -1.0
    done: float = -1.0
    records: object = None

    @property
    def shape(self):
        return tuple(int(s) for s in self.frames.shape)

    @property
    def nframes(self):
        return self.shape[0]

    @property
    def latency(self):
        return self.done - self.arrival


def record_capacity(T, H, W):
    """Records buffer: a detection needs a strict local maximum, so at most one per 2x2 block."""
    return max(16, (T * ((H + 1) // 2) * ((W + 1) // 2)))


def device_bytes(req: Request):
    T, H, W = req.shape
    return T * H * W * 2 + record_capacity(T, H, W) * 24 + 16


class Scheduler:
    """FIFO admission under a slot count and an HBM byte budget; executor-agnostic.

    An executor provides: slots (int), start(slot, req) and poll(slot) -> bool (True once
    the request on that slot has finished and its records are in req.records)."""

    def __init__(self, executor, hbm_budget: int, clock=time.perf_counter):
        self.ex = executor
        self.budget = int(hbm_budget)
        self.clock = clock
        self.in_use = 0
        self.peak_in_use = 0
        self.max_queue = 0

    def run(self, requests, idle_sleep=5e-5):
        reqs = sorted(requests, key=lambda r: r.arrival)
        for r in reqs:
            if device_bytes(r) > self.budget:
                raise ValueError(f"request {r.rid} needs {device_bytes(r)} bytes, above the HBM budget {self.budget}")
        waiting = collections.deque()
        free = list(range(self.ex.slots))
        running = {}  # slot -> request
        nxt = 0
        t0 = self.clock()
        done = 0
        while done < len(reqs):
            now = self.clock() - t0
            progressed = False
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                waiting.append(reqs[nxt])
                nxt += 1
            self.max_queue = max(self.max_queue, len(waiting))
            while waiting and free and self.in_use + device_bytes(waiting[0]) <= self.budget:
                r = waiting.popleft()
                slot = free.pop(0)
                self.in_use += device_bytes(r)
                self.peak_in_use = max(self.peak_in_use, self.in_use)
                r.admitted = self.clock() - t0
                self.ex.start(slot, r)
                running[slot] = r
                progressed = True
            for slot in list(running):
                if self.ex.poll(slot):
                    r = running.pop(slot)
                    r.done = self.clock() - t0
                    self.in_use -= device_bytes(r)
                    free.append(slot)
                    done += 1
                    progressed = True
            if not progressed:
                if nxt < len(reqs) and not running and not waiting:
                    time.sleep(max(0.0, min(reqs[nxt].arrival - (self.clock() - t0), 0.01)))
                else:
                    time.sleep(idle_sleep)
        return reqs


def report(reqs):
    lat = np.array([r.latency for r in reqs])
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    frames = sum(r.nframes for r in reqs)
    px = sum(int(np.prod(r.shape)) for r in reqs)
    return {
        "requests": len(reqs),
        "p50_ms": float(np.percentile(lat, 50) * 1e3),
        "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "frames_per_s": frames / span,
        "mpix_per_s": px / span / 1e6,
        "span_s": span,
    }


class GpuExecutor:
    """Slots = library contexts, each with its own CUDA stream."""

    def __init__(self, spec_json: str, blob: bytes, slots: int = 3, device=0):
        import torch

        from . import Localizer

        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.slots = slots
        self.locs = [Localizer(spec_json, blob) for _ in range(slots)]
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(slots)]
        self.state = [None] * slots
        # per-slot buffers, grown on demand and reused (no allocation on the request path
        # once they are large enough)
        self.d_out = [None] * slots
        self.h_out = [None] * slots
        self.h_n = [torch.empty(1, dtype=torch.int64, pin_memory=True) for _ in range(slots)]
        self.d_n = [torch.zeros(1, dtype=torch.int64, device=self.dev) for _ in range(slots)]

    def _buffers(self, slot, cap):
        torch = self.torch
        if self.d_out[slot] is None or self.d_out[slot].numel() < cap * 24:
            self.d_out[slot] = torch.empty(cap * 24, dtype=torch.uint8, device=self.dev)
            self.h_out[slot] = torch.empty(cap * 24, dtype=torch.uint8, pin_memory=True)
        return self.d_out[slot], self.h_out[slot]

    def warm(self, shapes, max_request=None):
        """Create each slot's workspace for the given frame sizes (and, if given, record buffers
        for the largest request shape (T, H, W)) before timing."""
        torch = self.torch
        for slot, (loc, st) in enumerate(zip(self.locs, self.streams)):
            for (H, W) in shapes:
                fr = torch.zeros((1, H, W), dtype=torch.uint16, device=self.dev)
                out = torch.empty(record_capacity(1, H, W) * 24, dtype=torch.uint8, device=self.dev)
                n = torch.zeros(1, dtype=torch.int64, device=self.dev)
                loc.localize_async(fr, 0.5, out, n, stream=st)
            if max_request is not None:
                self._buffers(slot, record_capacity(*max_request))
        torch.cuda.synchronize(self.dev)

    def start(self, slot, r: Request):
        torch = self.torch
        st = self.streams[slot]
        T, H, W = r.shape
        cap = record_capacity(T, H, W)
        d_out, _ = self._buffers(slot, cap)
        d_n, h_n = self.d_n[slot], self.h_n[slot]
        with torch.cuda.stream(st):
            d_frames = r.frames.to(self.dev, non_blocking=True)
        self.locs[slot].localize_async(d_frames, r.p_min, d_out[: cap * 24], d_n, gain=r.gain, offset=r.offset,
                                       gain_map=r.gain_map, offset_map=r.offset_map, stream=st)
        with torch.cuda.stream(st):
            h_n.copy_(d_n, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        self.state[slot] = {"req": r, "phase": 1, "ev": ev, "d_frames": d_frames, "d_out": d_out, "h_n": h_n}

    def poll(self, slot):
        torch = self.torch
        s = self.state[slot]
        if s is None or not s["ev"].query():
            return False
        if s["phase"] == 1:  # count known: copy exactly the records back
            n = int(s["h_n"][0])
            st = self.streams[slot]
            h_out = self.h_out[slot]
            with torch.cuda.stream(st):
                if n:
                    h_out[: n * 24].copy_(s["d_out"][: n * 24], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(st)
            s.update(phase=2, ev=ev, h_out=h_out, n=n)
            return False
        from . import RECORD_DTYPE

        r = s["req"]
        r.records = s["h_out"][: s["n"] * 24].numpy().view(RECORD_DTYPE).copy()
        self.state[slot] = None
        return True


class FakeExecutor:
    """Host-only executor with a fixed service time per frame (for testing the scheduler)."""

    def __init__(self, slots, s_per_frame, clock):
        self.slots = slots
        self.s_per_frame = s_per_frame
        self.clock = clock
        self.busy_until = [None] * slots
        self.reqs = [None] * slots
        self.concurrent_peak = 0

    def start(self, slot, r):
        self.busy_until[slot] = self.clock() + r.nframes * self.s_per_frame
        self.reqs[slot] = r
        self.concurrent_peak = max(self.concurrent_peak, sum(b is not None for b in self.busy_until))

    def poll(self, slot):
        if self.busy_until[slot] is not None and self.clock() >= self.busy_until[slot]:
            self.reqs[slot].records = np.zeros(0)
            self.busy_until[slot] = None
            return True
        return False


def poisson_arrivals(n, rate_per_s, rng):
    return np.cumsum(rng.exponential(1.0 / rate_per_s, n))

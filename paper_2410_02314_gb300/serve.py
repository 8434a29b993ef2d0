"""Serving loop: frame stacks of mixed sizes arrive over time and are localized with
continuous batching on one GPU.

* Weights and per-size workspaces stay resident: each slot is one library context (its own
  workspace and TMA descriptors, kept per frame size) driving its own CUDA stream.
* Admission: requests wait in arrival order and start as soon as a slot is free and their
  device memory fits the HBM budget next to what is already held.  The budget counts
  everything the serving loop holds on the device: every slot's resident workspaces (one
  per frame size a slot has run, reported by the library) and record buffers, plus, per
  running request, its frames and records; a request whose frame size is new to its slot
  is also charged the workspace the library will allocate for it.  The budget defaults to
  the device's free memory at the start of the run plus what the slots already hold, minus
  a reserve.  Requests that arrive while others run are admitted the moment a slot and
  memory free up, and their kernels interleave with the running ones on the device.
* Each request's records are the same alone and in the mix: every frame is computed
  independently and deterministically (no reduction depends on what else is on the GPU).
* A kernel that gave up on one of its bounded waits sets its context's error word; the
  executor reads the word with each request's record count and fails that request
  (Request.error) instead of returning incomplete records.
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
    error: str | None = None  # set when the request failed on the device
    slot: int = -1

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


def request_bytes(req: Request):
    """Device bytes a running request holds beyond its slot's resident state: its frames, its
    record buffer and its count."""
    T, H, W = req.shape
    return T * H * W * 2 + record_capacity(T, H, W) * 24 + 16


class Scheduler:
    """FIFO admission under a slot count and an HBM byte budget; executor-agnostic.

    An executor provides: slots (int); start(slot, req); poll(slot) -> bool (True once the
    request on that slot has finished: its records are in req.records, or req.error says why
    it failed); resident_bytes() (device bytes every slot holds between requests: workspaces
    and record buffers); plan_bytes(slot, shape) (workspace a request of that (T, H, W) shape
    adds on that slot: 0 if the slot holds one for H x W); and, for a budget derived from the
    device, memory_budget(reserve)."""

    def __init__(self, executor, hbm_budget: int | None = None, reserve: int = 4 << 30, clock=time.perf_counter):
        self.ex = executor
        self.budget = int(hbm_budget) if hbm_budget is not None else int(executor.memory_budget(reserve))
        self.clock = clock
        self.in_use = 0
        self.peak_in_use = 0
        self.max_queue = 0
        self.failed = 0

    def _need(self, slot, r):
        return request_bytes(r) + self.ex.plan_bytes(slot, r.shape)

    def _pick_slot(self, free, r):
        """A free slot that already holds the request's workspace, else the first free slot."""
        for k, slot in enumerate(free):
            if self.ex.plan_bytes(slot, r.shape) == 0:
                return k
        return 0

    def run(self, requests, idle_sleep=5e-5):
        reqs = sorted(requests, key=lambda r: r.arrival)
        base = self.ex.resident_bytes()
        for r in reqs:
            need = min(self._need(s, r) for s in range(self.ex.slots))
            if base + need > self.budget:
                raise ValueError(f"request {r.rid} needs {need} bytes next to the {base} resident, above the HBM "
                                 f"budget {self.budget}")
        waiting = collections.deque()
        free = list(range(self.ex.slots))
        running = {}  # slot -> request
        transient = 0  # bytes of the running requests
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
            while waiting and free:
                r = waiting[0]
                k = self._pick_slot(free, r)
                slot = free[k]
                plan = self.ex.plan_bytes(slot, r.shape)
                if self.ex.resident_bytes() + plan + transient + request_bytes(r) > self.budget:
                    break
                waiting.popleft()
                free.pop(k)
                transient += request_bytes(r)
                r.slot = slot
                r.admitted = self.clock() - t0
                self.ex.start(slot, r)  # allocates the new workspace, if any
                running[slot] = r
                self.in_use = self.ex.resident_bytes() + transient
                self.peak_in_use = max(self.peak_in_use, self.in_use)
                progressed = True
            for slot in list(running):
                if self.ex.poll(slot):
                    r = running.pop(slot)
                    r.done = self.clock() - t0
                    transient -= request_bytes(r)
                    self.in_use = self.ex.resident_bytes() + transient
                    self.failed += r.error is not None
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
        "failed": sum(r.error is not None for r in reqs),
    }


MAX_PLANS = 4  # frame sizes whose workspace a library context keeps (least recently used freed first)


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
        self.h_n = [torch.empty(2, dtype=torch.int64, pin_memory=True) for _ in range(slots)]
        # count (element 0) and the context's error word (low half of element 1)
        self.d_n = [torch.zeros(2, dtype=torch.int64, device=self.dev) for _ in range(slots)]

    def _buffers(self, slot, cap):
        torch = self.torch
        if self.d_out[slot] is None or self.d_out[slot].numel() < cap * 24:
            self.d_out[slot] = torch.empty(cap * 24, dtype=torch.uint8, device=self.dev)
            self.h_out[slot] = torch.empty(cap * 24, dtype=torch.uint8, pin_memory=True)
        return self.d_out[slot], self.h_out[slot]

    def warm(self, shapes, max_request=None):
        """Create each slot's workspace for the given request shapes (T, H, W), at most
        MAX_PLANS frame sizes, and, if given, record buffers for the largest request shape
        before timing."""
        torch = self.torch
        for slot, (loc, st) in enumerate(zip(self.locs, self.streams)):
            for (T, H, W) in shapes:
                fr = torch.zeros((T, H, W), dtype=torch.uint16, device=self.dev)
                out = torch.empty(record_capacity(T, H, W) * 24, dtype=torch.uint8, device=self.dev)
                n = torch.zeros(1, dtype=torch.int64, device=self.dev)
                loc.localize_async(fr, 0.5, out, n, stream=st)
            if max_request is not None:
                self._buffers(slot, record_capacity(*max_request))
        torch.cuda.synchronize(self.dev)

    def resident_bytes(self):
        """Workspaces every slot's context holds (the library's own count) and the slots'
        record buffers."""
        from . import sml_workspace_bytes

        ws = sum(sml_workspace_bytes(loc.ctx, 1, 1, 1)[2] for loc in self.locs)
        return ws + sum(0 if d is None else d.numel() for d in self.d_out)

    def plan_bytes(self, slot, shape):
        """Device bytes a request of shape (T, H, W) adds to what the slot keeps: the library's
        workspace for H x W if the slot's context holds none (the library's own figure; the
        plan it may free in exchange is not credited), and the growth of the slot's record
        buffer if the request needs a larger one."""
        from . import sml_workspace_bytes

        T, H, W = shape
        pb, res, _ = sml_workspace_bytes(self.locs[slot].ctx, T, H, W)
        have = 0 if self.d_out[slot] is None else self.d_out[slot].numel()
        return (0 if res else pb) + max(0, record_capacity(T, H, W) * 24 - have)

    def memory_budget(self, reserve):
        """The device's free memory now, plus what the slots already hold, minus `reserve`."""
        free, _ = self.torch.cuda.mem_get_info(self.dev)
        return free + self.resident_bytes() - reserve

    def start(self, slot, r: Request):
        from . import sml_error_word

        torch = self.torch
        st = self.streams[slot]
        T, H, W = r.shape
        cap = record_capacity(T, H, W)
        d_out, _ = self._buffers(slot, cap)
        d_n, h_n = self.d_n[slot], self.h_n[slot]
        with torch.cuda.stream(st):
            d_frames = r.frames.to(self.dev, non_blocking=True)
            d_n[1:].zero_()
        self.locs[slot].localize_async(d_frames, r.p_min, d_out[: cap * 24], d_n[:1], gain=r.gain, offset=r.offset,
                                       gain_map=r.gain_map, offset_map=r.offset_map, stream=st)
        # the context's error word after this request's kernels, next to its count
        sml_error_word(self.locs[slot].ctx, d_n[1:].view(torch.int32)[:1], stream=st)
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
            if int(s["h_n"][1]) != 0:
                return self._fail(slot, "a kernel gave up on a bounded wait; the request's records are incomplete")
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

    def _fail(self, slot, why):
        r = self.state[slot]["req"]
        r.error = why
        r.records = None
        self.state[slot] = None
        return True


class FakeExecutor:
    """Host-only executor with a fixed service time per frame (for testing the scheduler).
    It models the library's per-slot workspaces: a frame size new to a slot costs
    plan_cost(H, W) bytes, kept until the slot's MAX_PLANS-th newer size evicts it.
    fail_rids: requests whose device work reports an error."""

    def __init__(self, slots, s_per_frame, clock, plan_cost=lambda H, W: 0, fail_rids=()):
        self.slots = slots
        self.s_per_frame = s_per_frame
        self.clock = clock
        self.plan_cost = plan_cost
        self.fail_rids = set(fail_rids)
        self.busy_until = [None] * slots
        self.reqs = [None] * slots
        self.plans = [collections.OrderedDict() for _ in range(slots)]  # (H, W) -> bytes, LRU first
        self.concurrent_peak = 0

    def resident_bytes(self):
        return sum(sum(p.values()) for p in self.plans)

    def plan_bytes(self, slot, shape):
        _, H, W = shape
        return 0 if (H, W) in self.plans[slot] else self.plan_cost(H, W)

    def start(self, slot, r):
        _, H, W = r.shape
        p = self.plans[slot]
        if (H, W) in p:
            p.move_to_end((H, W))
        else:
            if len(p) >= MAX_PLANS:
                p.popitem(last=False)
            p[(H, W)] = self.plan_cost(H, W)
        self.busy_until[slot] = self.clock() + r.nframes * self.s_per_frame
        self.reqs[slot] = r
        self.concurrent_peak = max(self.concurrent_peak, sum(b is not None for b in self.busy_until))

    def poll(self, slot):
        if self.busy_until[slot] is not None and self.clock() >= self.busy_until[slot]:
            r = self.reqs[slot]
            if r.rid in self.fail_rids:
                r.error = "injected device error"
            else:
                r.records = np.zeros(0)
            self.busy_until[slot] = None
            return True
        return False


def poisson_arrivals(n, rate_per_s, rng):
    return np.cumsum(rng.exponential(1.0 / rate_per_s, n))

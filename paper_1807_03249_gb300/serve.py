"""Continuous-batching request loop for StyleBlit stylisation.

Requests (a target guide in pinned host memory, an exemplar id and the method's
parameters: levels, threshold, seed; one blend radius per server) arrive over
time.  The loop keeps every exemplar's guide, style and look-up table resident
on the device and admits waiting requests in arrival order whenever a slot (a
CUDA stream) is free and their device buffers fit the HBM budget.  Each
admitted group runs as one sb_stylize_batch launch between its host-to-device
and device-to-host copies on its slot's stream, so groups on different slots
overlap on the device, and requests arriving meanwhile join the next group.

The scheduling core (`Scheduler`) is plain Python and knows nothing of CUDA;
`Server` binds it to the library.  Every result is exactly what sb_stylize
gives for that request alone (the batch kernel is bit-identical per frame).
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Callable

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float            # seconds, on the loop's clock
    exemplar: int
    guide: object             # host tensor [H, W, C] (pinned for real overlap)
    levels: int
    threshold: int
    seed: int
    nbytes: int = 0           # device bytes while in flight (guide + RGBA8 output)
    admitted: float | None = None
    done: float | None = None
    out: object = None        # host RGBA8 result (allocated pinned when None)

    @property
    def pixels(self) -> int:
        return int(self.guide.shape[0]) * int(self.guide.shape[1])


class Scheduler:
    """Admission by slots and byte budget, FIFO, groups of at most max_batch."""

    def __init__(self, budget_bytes: int, slots: int, max_batch: int):
        self.budget = int(budget_bytes)
        self.slots = int(slots)
        self.max_batch = int(max_batch)
        self.waiting: collections.deque[Request] = collections.deque()
        self.in_use = 0
        self.peak_in_use = 0
        self.free_slots = list(range(self.slots))

    def submit(self, req: Request):
        if req.nbytes > self.budget:
            raise ValueError(f"request {req.rid} needs {req.nbytes} bytes, budget {self.budget}")
        self.waiting.append(req)

    def next_group(self):
        """A (slot, requests) group to launch now, or None."""
        if not self.free_slots or not self.waiting:
            return None
        group, nbytes = [], 0
        while (self.waiting and len(group) < self.max_batch and
               self.in_use + nbytes + self.waiting[0].nbytes <= self.budget):
            r = self.waiting.popleft()
            group.append(r)
            nbytes += r.nbytes
        if not group:
            return None  # the head does not fit yet: wait for memory (FIFO, no overtaking)
        self.in_use += nbytes
        self.peak_in_use = max(self.peak_in_use, self.in_use)
        return self.free_slots.pop(0), group

    def finish(self, slot: int, group):
        self.in_use -= sum(r.nbytes for r in group)
        self.free_slots.append(slot)


def latency_summary(reqs, wall_s: float) -> dict:
    lat = np.array([r.done - r.arrival for r in reqs]) * 1e3
    px = sum(r.pixels for r in reqs)
    return {"requests": len(reqs), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "frames_per_s": len(reqs) / wall_s, "mpixel_per_s": px / wall_s / 1e6,
            "wall_s": wall_s}


class Server:
    """The loop bound to one CUDA device through the StyleBlit library."""

    def __init__(self, device, radius: int, budget_bytes: int = 40 << 30, slots: int = 4,
                 max_batch: int = 16):
        import torch

        from . import MAX_BATCH
        self.torch = torch
        self.device = torch.device(device)
        self.radius = radius
        self.sched = Scheduler(budget_bytes, slots, min(max_batch, MAX_BATCH))
        self.streams = [torch.cuda.Stream(self.device) for _ in range(slots)]
        self.exemplars = {}
        self.inflight = []  # (event, slot, group, keep-alive tensors)

    def add_exemplar(self, ex_id: int, guide, style, key_bits: int):
        """Uploads an exemplar and builds its table; both stay resident."""
        from . import build_lut
        t = self.torch
        g = t.from_numpy(guide.view(np.int16) if guide.dtype == np.uint16 else guide)
        gd = g.to(self.device)
        sd = t.from_numpy(style).to(self.device)
        self.exemplars[ex_id] = (gd, sd, build_lut(gd, key_bits))

    def device_bytes(self, guide) -> int:
        h, w = int(guide.shape[0]), int(guide.shape[1])
        return guide.element_size() * guide.numel() + 4 * h * w

    def submit(self, req: Request):
        req.nbytes = self.device_bytes(req.guide)
        self.sched.submit(req)

    def _launch(self, slot: int, group, now: Callable[[], float]):
        from . import BatchFrame, stylize_batch
        t = self.torch
        s = self.streams[slot]
        keep = []
        with t.cuda.stream(s):
            frames = []
            for r in group:
                g = t.empty(r.guide.shape, dtype=r.guide.dtype, device=self.device)
                g.copy_(r.guide, non_blocking=True)
                _, sd, lut = self.exemplars[r.exemplar]
                frames.append(BatchFrame(g, lut, sd, r.levels, r.threshold, r.seed))
                keep.append(g)
            stylize_batch(frames, self.radius, stream=s)
            for r, f in zip(group, frames):
                if r.out is None:
                    r.out = t.empty(f.out.shape, dtype=t.uint8, pin_memory=True)
                r.out.copy_(f.out, non_blocking=True)
                keep.append(f.out)
            ev = t.cuda.Event()
            ev.record(s)
        t_adm = now()
        for r in group:
            r.admitted = t_adm
        self.inflight.append((ev, slot, group, keep))

    def poll(self, now: Callable[[], float]):
        """Retires finished groups (frees their slot and bytes); returns their requests."""
        done, still = [], []
        for item in self.inflight:
            ev, slot, group, keep = item
            if ev.query():
                t_done = now()
                for r in group:
                    r.done = t_done
                self.sched.finish(slot, group)
                done.extend(group)
            else:
                still.append(item)
        self.inflight = still
        return done

    def pump(self, now: Callable[[], float]):
        """Launches every group the scheduler admits right now."""
        while True:
            nxt = self.sched.next_group()
            if nxt is None:
                return
            self._launch(*nxt, now=now)

    def run(self, requests, real_time: bool = True, timeout_s: float = 600.0):
        """Feeds requests at their arrival times (seconds from the start) and
        serves them all; returns the finished requests in completion order."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        finished = []
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731
        n = len(pending)
        while len(finished) < n:
            t = now()
            if t > timeout_s:
                raise TimeoutError(f"served {len(finished)} of {n} requests in {timeout_s} s")
            while pending and (not real_time or pending[0].arrival <= t):
                r = pending.popleft()
                if not real_time:
                    r.arrival = t
                self.submit(r)
            finished.extend(self.poll(now))
            self.pump(now)
        self.torch.cuda.synchronize(self.device)
        return finished, now()

"""Continuous-batching request loop for StyleBlit stylisation.

Requests (a target guide in pinned host memory, an exemplar id and the method's
parameters: levels, threshold, seed; one blend radius per server) arrive over
time.  The loop keeps every exemplar's guide, style and look-up table resident
on the device and admits waiting requests in arrival order whenever a slot (a
CUDA stream) is free and their device buffers fit the HBM budget.  Each
admitted group runs as one sb_stylize_batch launch between its host-to-device
and device-to-host copies on its slot's stream, so groups on different slots
overlap on the device, and requests arriving meanwhile join the next group.
Results return smallest first and a request is done as soon as its own result
is back on the host.

Each slot owns one device buffer (its arena) that holds its group's guides and
outputs, so serving makes no device allocation per request: an arena grows in
64 MiB steps only when a group larger than any before arrives on that slot, and
`Server.reserve` sizes them before serving starts.  The byte budget bounds the
bytes of the requests in flight.

The scheduling core (`Scheduler`) is plain Python and knows nothing of CUDA;
`Server` binds it to the library.  Every result is exactly what sb_stylize
gives for that request alone (the batch kernel is bit-identical per frame).
"""
from __future__ import annotations

import collections
import dataclasses
import gc
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


class SlotArena:
    """One slot's device buffer.  A group's guides and RGBA8 outputs are carved
    from it as contiguous [H, W, C] views at 256-byte boundaries, and it grows
    in 64 MiB steps to the largest group the slot has held.  The caller grows
    or reuses it only while the slot is free (its previous group's work done)."""

    ALIGN = 256
    STEP = 64 << 20

    def __init__(self, torch, device):
        self.torch, self.device = torch, device
        self.buf = None
        self._typed = {}
        self._off = 0

    @classmethod
    def aligned(cls, n: int) -> int:
        return (n + cls.ALIGN - 1) // cls.ALIGN * cls.ALIGN

    @classmethod
    def request_bytes(cls, guide) -> int:
        """Arena bytes of one request: its guide and RGBA8 output, each aligned."""
        h, w = int(guide.shape[0]), int(guide.shape[1])
        return cls.aligned(guide.element_size() * guide.numel()) + cls.aligned(4 * h * w)

    @property
    def capacity(self) -> int:
        return 0 if self.buf is None else self.buf.numel()

    def ensure(self, nbytes: int):
        if self.capacity >= nbytes:
            return
        cap = max(1, -(-nbytes // self.STEP)) * self.STEP
        self.buf, self._typed = None, {}
        self.buf = self.torch.empty(cap, dtype=self.torch.uint8, device=self.device)

    def start_group(self, nbytes: int):
        """Makes room for a group of nbytes and carves from the start again."""
        self.ensure(nbytes)
        self._off = 0

    def carve(self, dtype, shape):
        """The next contiguous view of the given dtype and [H, W, C] shape."""
        if dtype not in self._typed:
            self._typed[dtype] = self.buf.view(dtype)
        a = self._typed[dtype]
        size = a.element_size()
        nbytes = size * shape[0] * shape[1] * shape[2]
        if self._off + nbytes > self.capacity:
            raise ValueError(f"arena of {self.capacity} bytes cannot hold {self._off + nbytes}")
        v = a.as_strided(tuple(shape), (shape[1] * shape[2], shape[2], 1), self._off // size)
        self._off += self.aligned(nbytes)
        return v


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
        # per slot: one device buffer that holds its group's guides and outputs
        self.arenas = [SlotArena(torch, self.device) for _ in range(slots)]
        self.exemplars = {}
        self.inflight = []  # (slot, group, per-request events)
        self.max_loop_gap_s = 0.0

    def reserve(self, nbytes_per_slot: int):
        """Sizes every slot's arena for groups of up to nbytes_per_slot bytes
        now, so that serving allocates no device memory afterwards."""
        for slot in self.sched.free_slots:
            self.arenas[slot].ensure(nbytes_per_slot)

    def add_exemplar(self, ex_id: int, guide, style, key_bits: int):
        """Uploads an exemplar and builds its table; both stay resident."""
        from . import build_lut
        t = self.torch
        g = t.from_numpy(guide.view(np.int16) if guide.dtype == np.uint16 else guide)
        gd = g.to(self.device)
        sd = t.from_numpy(style).to(self.device)
        self.exemplars[ex_id] = (gd, sd, build_lut(gd, key_bits))

    def device_bytes(self, guide) -> int:
        """Device bytes of one request in its slot's arena: the guide and the
        RGBA8 output, each 256-byte aligned."""
        return SlotArena.request_bytes(guide)

    def submit(self, req: Request):
        req.nbytes = self.device_bytes(req.guide)
        self.sched.submit(req)

    def _launch(self, slot: int, group, now: Callable[[], float]):
        from . import BatchFrame, stylize_batch
        t = self.torch
        s = self.streams[slot]
        arena = self.arenas[slot]
        arena.start_group(sum(r.nbytes for r in group))
        with t.cuda.stream(s):
            frames = []
            for r in group:
                src = r.guide if r.guide.dim() == 3 else r.guide.unsqueeze(-1)
                h, w = int(src.shape[0]), int(src.shape[1])
                g = arena.carve(src.dtype, tuple(src.shape))
                g.copy_(src, non_blocking=True)
                o = arena.carve(t.uint8, (h, w, 4))
                _, sd, lut = self.exemplars[r.exemplar]
                frames.append(BatchFrame(g, lut, sd, r.levels, r.threshold, r.seed, out=o))
            stylize_batch(frames, self.radius, stream=s)
            # results go back smallest first, each followed by its own event, so
            # a small request is done as soon as its own copy is; the last event
            # marks the group's (and the slot's) end
            evs = [None] * len(group)
            for i in sorted(range(len(group)), key=lambda i: group[i].pixels):
                r, f = group[i], frames[i]
                if r.out is None:
                    r.out = t.empty(f.out.shape, dtype=t.uint8, pin_memory=True)
                r.out.copy_(f.out, non_blocking=True)
                evs[i] = t.cuda.Event()
                evs[i].record(s)
        t_adm = now()
        for r in group:
            r.admitted = t_adm
            r.done = None
        self.inflight.append((slot, group, evs))

    def poll(self, now: Callable[[], float]):
        """Stamps each request whose result is back on the host, retires
        groups whose results all are (frees their slot and bytes) and returns
        the requests of those groups."""
        done, still = [], []
        for item in self.inflight:
            slot, group, evs = item
            for r, ev in zip(group, evs):
                if r.done is None and ev.query():
                    r.done = now()
            if all(r.done is not None for r in group):
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
        serves them all; returns the finished requests in completion order.
        The cyclic garbage collector is paused while the loop runs (after one
        collection before it), so no collection pass lands inside a request's
        latency.  `max_loop_gap_s` records the longest time between two
        passes of the loop: a stall of the host side (the process not
        running, or a blocking call) shows there."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        finished = []
        gc_was_enabled = gc.isenabled()
        gc.collect()
        gc.disable()
        try:
            t0 = time.perf_counter()
            now = lambda: time.perf_counter() - t0  # noqa: E731
            n = len(pending)
            self.max_loop_gap_s = 0.0
            t_prev = 0.0
            while len(finished) < n:
                t = now()
                self.max_loop_gap_s = max(self.max_loop_gap_s, t - t_prev)
                t_prev = t
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
        finally:
            if gc_was_enabled:
                gc.enable()

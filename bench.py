"""Throughput benchmark of the GB300 StyleBlit hot path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload 1080p|4k]
                    [--impl reference]

A step stylises `frames_per_step` distinct target frames of the workload in
one sb_stylize_batch launch (Algorithm 2 assignment + Section 3.2 vote, fused,
every tile of every frame in one grid) against a device-resident exemplar and
look-up table.  The frames' guides and outputs exceed the L2 cache, so every
step reads its inputs from HBM.  Steps are replayed from a CUDA graph so host
launch overhead cannot starve the GPU.  The same frames launched one
sb_stylize per frame are timed too (`per_frame_launch`).  Prints one JSON line
on rank 0.

--impl reference times the CPU oracle (plain C, all host cores) on a
bounded sample of the same workload and prints the same JSON line.
Under torchrun each rank stylises its own frames (weak scaling, no data-path
collective); only timing uses a barrier and a max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

L2_BYTES = 126 * 1024 * 1024
FRAMES_PER_STEP = 24
E2E_GROUP = 4        # frames per batch launch on the end-to-end leg (24 frames: two groups per stream)
METRIC = "Mpixel/s stylized (1080p/4K, blend on) and % HBM roofline; served p50/p99 latency"


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--workload", choices=["1080p", "4k"], default="1080p")
    p.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    p.add_argument("--e2e-steps", type=int, default=20)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-served", action="store_true")
    p.add_argument("--no-4k", action="store_true",
                   help="skip the 3840x2160 UV workload (batched and single-frame) on the line")
    p.add_argument("--no-uneven", action="store_true",
                   help="skip the uneven batch (64 mixed-size frames, 8 exemplars)")
    p.add_argument("--profile-once", action="store_true",
                   help="build the step's frames and launch sb_stylize_batch twice, then "
                        "sb_lookup_only_batch twice, no timing (a fixed launch sequence for ncu "
                        "captures)")
    p.add_argument("--single-frames", type=int, default=0,
                   help="with --profile-once: then this many sb_stylize calls, one per frame of the "
                        "step (the single-frame path), before the lookup-only launches")
    p.add_argument("--schedule", default="0,0,0,0",
                   help="with --profile-once: the batch schedule as persistent,largest_first,"
                        "interleave_rows,tile_rows (the bench line's config.schedule)")
    return p.parse_args()


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def make_workload(name: str, n_frames: int, rank: int = 0):
    """Exemplar + `n_frames` distinct target guides (a few generated fields,
    each shifted cyclically by seeded offsets)."""
    base = 3 if name == "1080p" else 2
    seed0 = rank_frame_seed(name, rank)
    w = synth.workload_1080p(base, seed0) if name == "1080p" else synth.workload_4k_uv(base, seed0)
    rng = np.random.default_rng(seed0)
    frames = []
    for i in range(n_frames):
        g = w.frames[i % base].guide
        dy, dx = int(rng.integers(0, g.shape[0])), int(rng.integers(0, g.shape[1]))
        frames.append(np.ascontiguousarray(np.roll(g, (dy, dx), axis=(0, 1))))
    return w, frames


def rank_frame_seed(name: str, rank: int) -> int:
    """Seed of rank `rank`'s frames: ranks stylise disjoint frames (weak
    scaling; frames are independent, so there is no data-path exchange)."""
    return (2000 if name == "1080p" else 3000) + 100 * rank


def max_over_ranks(ms: float, world: int, device=None) -> float:
    """The slowest rank's time (the job ends when every rank has finished)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, px_per_step_per_rank: int, steps: int, ms: float) -> float:
    """Whole-job Mpixel/s: every rank's pixels over the slowest rank's time."""
    return world * px_per_step_per_rank * steps / (ms / 1e3) / 1e6


def algorithmic_bytes(w, frame) -> dict:
    H, W, C = frame.shape
    px = H * W
    guide_b = px * C * frame.dtype.itemsize
    out_b = px * 4
    ex = w.exemplar
    ex_b = ex.style.nbytes + ex.guide.nbytes + 4 * (1 << (ex.guide.shape[2] * ex.lut_bits))
    return dict(pixels=px, frame_bytes=guide_b + out_b, exemplar_bytes=ex_b)


def _code_only(text: str) -> str:
    """C++ source without comments and with whitespace runs collapsed."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash() -> str:
    """Hash of the code the profiled batch kernel is compiled from (the frame
    kernels' header, the shared device helpers and the per-format translation
    units; comments and layout excluded), so committed counters go stale when
    the code changes."""
    d = os.path.join(ROOT, "paper_1807_03249_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        if f in ("sb_frame.cuh", "sb_internal.cuh", "sb_nn.cuh") or (f.startswith("sb_frame_c") and f.endswith(".cu")):
            h.update(_code_only(open(os.path.join(d, f)).read()).encode())
    return h.hexdigest()[:16]


def schedule_tag(sched: dict) -> str:
    """The schedule as the launch sees it: with rows interleaved every frame
    has the same tile grid, so largest-first ordering changes nothing."""
    keys = ("persistent", "interleave_rows", "tile_rows") if sched.get("interleave_rows") else \
        ("persistent", "largest_first", "interleave_rows", "tile_rows")
    return ",".join(f"{k}={int(sched.get(k, 0))}" for k in keys)


def profiled_counters(workload: str, sched: dict) -> dict:
    """Counters of one batch launch from the committed ncu summary, if it was
    taken on the current kernel sources under the same schedule (else {})."""
    path = os.path.join(ROOT, "profiles", f"sb_stylize_batch_{workload}_traffic.txt")
    if not os.path.exists(path):
        return {}
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_source_hash") != kernel_source_hash():
        return {}
    if kv.get("schedule") != schedule_tag(sched):
        return {}
    out = {}
    for k in ("dram_bytes_per_launch", "warp_instructions_per_launch"):
        try:
            out[k] = float(kv[k])
        except (KeyError, ValueError):
            pass
    return out


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.samples = []
        self.proc = None
        self.t0 = self.t1 = None
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "100"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append((time.monotonic(), parts))

    def mark(self, start: bool):
        if start:
            self.t0 = time.monotonic()
        else:
            self.t1 = time.monotonic()

    def stop(self) -> dict:
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        inside = [p for t, p in self.samples if self.t0 and self.t1 and self.t0 <= t <= self.t1]
        window = "timed"
        if not inside:
            inside = [p for _, p in self.samples[-5:]]
            window = "after-timed (timed region shorter than the sampling period)"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(p[1]) for p in inside if num(p[1]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for p in inside:
            for n, v in zip(names, p[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": num(inside[0][2]), "power_w_max": max(
                    (num(p[3]) or 0.0) for p in inside),
                "reasons": sorted(reasons), "samples": len(inside), "window": window}


# ---------------------------------------------------------------------------
# CPU oracle baseline
# ---------------------------------------------------------------------------

def cpu_oracle_run(w, frames, steps: int = 0, warmup: int = 1, budget_s: float = 12.0,
                   threads: int = 0):
    """Times the oracle (assignment + RGBA8 vote, every host core) on bands of
    rows of the workload's frames.  Table entries a band needs are filled in
    untimed warm-up passes first (the GPU also runs with a resident table).
    steps > 0: `warmup` untimed then `steps` timed bands, the band height
    chosen so the timed part takes about `budget_s`; steps == 0: as many
    64-row bands as fit in `budget_s`.  threads: oracle threads (0: every core)."""
    import oracle
    ex = w.exemplar
    all_cores = os.cpu_count() or 1
    cores = threads or all_cores
    lut = oracle.new_lut(ex.guide.shape[2], ex.lut_bits)
    full = [np.ascontiguousarray(f) for f in frames[:2]]

    n_bands = 4  # a fixed set of bands: the warm-up fills every table entry they need

    def run_band(k, rows, n_threads=cores):
        g = full[k % len(full)]
        y0 = ((k % n_bands) * (g.shape[0] // n_bands)) % max(1, g.shape[0] - rows + 1)
        band = np.ascontiguousarray(g[y0:y0 + rows])
        t = time.perf_counter()
        a, _ = oracle.assign(band, ex.guide, ex.lut_bits, w.levels, w.threshold, w.seed + k % 2,
                             lut=lut, n_threads=n_threads)
        oracle.blend_rgba8(a, ex.style, w.blend_radius, n_threads=n_threads)
        return time.perf_counter() - t, band.shape[0] * band.shape[1]

    for k in range(max(n_bands, warmup)):  # untimed: fills the table entries bands need
        run_band(k, 64, all_cores)
    t64, _ = run_band(0, 64)  # table resident now: time of one 64-row band
    rows = 64
    if steps > 0:
        rows = int(max(1, min(64, 64 * budget_s / max(1e-9, steps * t64))))
    times, px, n = [], 0, 0
    t_start = time.perf_counter()
    while True:
        dt, p = run_band(n, rows)
        times.append(dt)
        px += p
        n += 1
        if steps > 0 and n >= steps:
            break
        if steps == 0 and time.perf_counter() - t_start > budget_s:
            break
    total = sum(times)
    return {"value": px / total / 1e6, "unit": "Mpixel/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} steps over {n_bands} fixed bands of {rows} rows x "
                      f"{full[0].shape[1]} px of the {w.name} "
                      f"frames, assignment + r={w.blend_radius} vote, table entries filled "
                      f"in untimed warm-up passes",
            "seconds": total, "ms_per_step": 1e3 * total / n, "steps": n}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w, frames = make_workload(args.workload, 2)
    r = cpu_oracle_run(w, frames, steps=args.steps, warmup=args.warmup, budget_s=90.0)
    H, W = frames[0].shape[:2]
    line = {"metric": METRIC, "value": r["value"], "unit": "Mpixel/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": w.name, "frame": f"{W}x{H}", "levels": w.levels,
                       "threshold": w.threshold, "blend": f"{2 * w.blend_radius + 1}x"
                       f"{2 * w.blend_radius + 1}",
                       "step": "one band of rows of a frame (see cpu_baseline.sample)"},
            "cpu_baseline": {k: r[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": r["value"], "unit": "Mpixel/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_1807_03249_gb300 as sb

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    def barrier():
        if world > 1:
            dist.barrier()

    w, frames = make_workload(args.workload, FRAMES_PER_STEP, rank)
    ex = w.exemplar
    H, W = frames[0].shape[:2]
    ab = algorithmic_bytes(w, frames[0])

    def to_dev(a):
        if a.dtype == np.uint16:
            a = a.view(np.int16)
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    g_src, style = to_dev(ex.guide), to_dev(ex.style)
    g_tgt = [to_dev(f) for f in frames]
    outs = [torch.empty((H, W, 4), dtype=torch.uint8, device=dev) for _ in frames]
    step_bytes = sum(t.numel() * t.element_size() for t in g_tgt) + sum(o.numel() for o in outs)
    assert step_bytes > L2_BYTES, "a step's inputs must exceed L2"

    stream = torch.cuda.Stream(dev)
    # exemplar preparation (A1, once per exemplar), timed separately
    torch.cuda.synchronize()
    t_lut = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            lut = sb.build_lut(g_src, ex.lut_bits, stream=stream)
            e1.record(stream)
        stream.synchronize()
        t_lut.append(e0.elapsed_time(e1))
        if _ < 2:
            lut.destroy()

    batch = [sb.BatchFrame(g_tgt[i], lut, style, w.levels, w.threshold, w.seed + i, out=outs[i])
             for i in range(FRAMES_PER_STEP)]

    # the launch schedule: the one sb_autotune_batch picks for this batch
    # (outputs are the same under every schedule)
    tuned, _ = sb.autotune_batch(batch, w.blend_radius, reps=5, stream=stream)
    torch.cuda.synchronize()

    def step_batch():
        sb.stylize_batch(batch, w.blend_radius, stream=stream, schedule=tuned)

    def step_frames():
        for i in range(FRAMES_PER_STEP):
            sb.stylize(g_tgt[i], g_src, style, lut, w.levels, w.threshold, w.blend_radius,
                       w.seed + i, out=outs[i], stream=stream)

    def capture(fn):
        # first call outside capture (per-kernel attribute set-up), then capture
        with torch.cuda.stream(stream):
            fn()
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            fn()
        torch.cuda.synchronize()
        return g

    def time_graph(g, steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(steps):
                g.replay()
            e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return max_over_ranks(e0.elapsed_time(e1), world, dev)


    graph = capture(step_batch)
    graph_frames = capture(step_frames)
    for _ in range(max(3, args.warmup)):
        with torch.cuda.stream(stream):
            graph.replay()
            graph_frames.replay()
    torch.cuda.synchronize()

    gpu_id = None
    try:
        gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
        gpu_id = gpu_id if gpu_id.startswith("GPU-") else "GPU-" + gpu_id
    except Exception:
        gpu_id = None
    sampler = ClockSampler(gpu_id)
    time.sleep(0.3)

    sampler.mark(True)
    ms = time_graph(graph, args.steps)
    sampler.mark(False)
    clocks = sampler.stop()
    ms_per_step = ms / args.steps
    px_step = FRAMES_PER_STEP * H * W
    value = job_throughput(world, px_step, args.steps, ms)
    pf_steps = max(3, min(args.steps, 300))
    ms_pf = time_graph(graph_frames, pf_steps)
    # every schedule of the same batch (one CTA per tile or persistent; frame
    # order or tile rows interleaved across the frames)
    by_schedule = {}
    for rows in (32, 16, 64):
        for pers in (0, 1):
            for il in (0, 1):
                sc = {"persistent": pers, "largest_first": 0, "interleave_rows": il,
                      "tile_rows": rows}
                gs_ = capture(lambda: sb.stylize_batch(batch, w.blend_radius, stream=stream,
                                                       schedule=sc))
                for _ in range(3):
                    with torch.cuda.stream(stream):
                        gs_.replay()
                by_schedule[f"tile_rows={rows},persistent={pers},interleave_rows={il}"] = \
                    time_graph(gs_, pf_steps) / pf_steps
                del gs_

    # the lookup-only comparator (Section 4, texture mapping) on the same frames:
    # one short launch per frame spread over four streams (forked from and
    # joined back to the step's stream) so their ramps and tails overlap; beside
    # it, one sb_lookup_only_batch launch per step
    lk_frames = [sb.BatchFrame(g_tgt[i], lut, style, w.levels, w.threshold, 0, out=outs[i])
                 for i in range(FRAMES_PER_STEP)]

    def step_lookup_batch():
        sb.lookup_only_batch(lk_frames)

    lk_streams = [torch.cuda.Stream(dev) for _ in range(4)]

    def step_lookup():
        cur = torch.cuda.current_stream()
        fork = torch.cuda.Event()
        fork.record(cur)
        for st_ in lk_streams:
            st_.wait_event(fork)
        for i in range(FRAMES_PER_STEP):
            sb.lookup_only(g_tgt[i], g_src, style, lut, out=outs[i],
                           stream=lk_streams[i % len(lk_streams)])
        for st_ in lk_streams:
            join = torch.cuda.Event()
            join.record(st_)
            cur.wait_event(join)

    lk_bytes = FRAMES_PER_STEP * ab["frame_bytes"]
    hbm_peak = measured_peaks().get("hbm_gbs") or 6800.0

    def lookup_line(ms):
        return {"value": job_throughput(world, px_step, pf_steps, ms), "unit": "Mpixel/s",
                "ms_per_step": ms / pf_steps,
                "hbm_frac": lk_bytes / (ms / pf_steps / 1e3) / 1e9 / hbm_peak}

    lookup = lookup_line(time_graph(capture(step_lookup), pf_steps))
    lookup["what"] = ("C_T[p] = C_S[LUT(G_T[p])] per pixel, one sb_lookup_only launch per frame "
                      "over 4 streams")
    lookup["batched"] = lookup_line(time_graph(capture(step_lookup_batch), pf_steps))
    lookup["batched"]["what"] = "every frame of the step in one sb_lookup_only_batch launch"
    per_frame = {"value": job_throughput(world, px_step, pf_steps, ms_pf), "unit": "Mpixel/s",
                 "ms_per_step": ms_pf / pf_steps, "steps": pf_steps,
                 "launch": "CUDA graph of frames_per_step sb_stylize kernels (one per frame)"}

    # end to end through the host-buffer batch call: groups of E2E_GROUP frames
    # are copied in from pinned memory, stylised by one batch launch and copied
    # out, consecutive groups on three streams so copies overlap kernels
    host_in = [torch.from_numpy(f.view(np.int16) if f.dtype == np.uint16 else f).pin_memory()
               for f in frames]
    host_out = [torch.empty((H, W, 4), dtype=torch.uint8).pin_memory() for _ in frames]
    staging = {}
    e2e_streams = [torch.cuda.Stream(dev) for _ in range(3)]
    seeds = [w.seed + i for i in range(FRAMES_PER_STEP)]

    def e2e_step():
        sb.stylize_batch_host(host_in, lut, style, w.levels, w.threshold, seeds, w.blend_radius,
                              host_out, group=E2E_GROUP, streams=e2e_streams, staging=staging)

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        x0.record(stream)
    for st_ in e2e_streams:
        st_.wait_event(x0)
    for _ in range(args.e2e_steps):
        e2e_step()
    for st_ in e2e_streams:
        ev = torch.cuda.Event()
        ev.record(st_)
        stream.wait_event(ev)
    with torch.cuda.stream(stream):
        x1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_e2e = max_over_ranks(x0.elapsed_time(x1), world, dev)
    e2e_value = job_throughput(world, px_step, args.e2e_steps, ms_e2e)
    h2d = sum(f.nbytes for f in frames)
    d2h = sum(o.numel() for o in host_out)
    copy_ceiling = copies_only(dev, host_in, host_out, staging, e2e_streams, stream)

    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    kernel_s = ms_per_step / 1e3  # one batch launch per step
    alg = FRAMES_PER_STEP * ab["frame_bytes"] + ab["exemplar_bytes"]
    achieved = alg / kernel_s / 1e9
    counters = profiled_counters(args.workload, tuned)
    traffic = counters.get("dram_bytes_per_launch")
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = peaks.get("sm_max_mhz") or 2070.0
    issue_peak = sm_count * 4 * sm_mhz * 1e6  # warp instructions per second
    inst = counters.get("warp_instructions_per_launch")
    issue = {"bound": "issue", "unit": "warp instructions/s", "peak": issue_peak,
             "peak_rule": f"{sm_count} SMs x 4 issue slots x {sm_mhz:.0f} MHz",
             "achieved": inst / kernel_s if inst else None,
             "frac": inst / kernel_s / issue_peak if inst else None,
             "instructions_per_launch": inst}

    line = {"metric": METRIC, "value": value, "unit": "Mpixel/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": w.name, "frame": f"{W}x{H}", "frames_per_step":
                       FRAMES_PER_STEP, "levels": w.levels, "threshold": w.threshold,
                       "blend": f"{2 * w.blend_radius + 1}x{2 * w.blend_radius + 1}",
                       "exemplar": f"{ex.guide.shape[1]}x{ex.guide.shape[0]}, LUT "
                                   f"{ex.lut_bits} bits/channel",
                       "l2": f"no flush: each step reads {step_bytes / 2**20:.0f} MiB of "
                             f"distinct guides and outputs (> {L2_BYTES // 2**20} MiB L2)",
                       "launch": "CUDA graph of one sb_stylize_batch launch over all "
                                 "frames_per_step frames, schedule picked by "
                                 "sb_autotune_batch",
                       "schedule": tuned,
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic,
                         "kernel": f"batch_kernel{'_persistent' if tuned.get('persistent') else ''}"
                                   f"<{ex.guide.shape[2]},{ex.guide.dtype.itemsize * 8},"
                                   f"{w.blend_radius},{int(tuned.get('tile_rows') or 32)}> "
                                   f"(sb_stylize_batch)",
                         "peak_source": f"{peak_src} copy bandwidth",
                         "algorithmic_bytes_per_launch": alg,
                         "frame_only_frac": FRAMES_PER_STEP * ab["frame_bytes"] / kernel_s
                         / 1e9 / hbm,
                         "kernel_us": kernel_s * 1e6,
                         "bytes_rule": "24 frames x (guide in + RGBA8 out) + exemplar "
                                       "(style + guide + table) once per launch"},
            "e2e": {"value": e2e_value, "unit": "Mpixel/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
                    "api": f"stylize_batch_host (pinned host in/out), groups of {E2E_GROUP} "
                           "frames over 3 streams",
                    "copies_only": {
                        "value": job_throughput(world, px_step, 1, copy_ceiling["ms"]),
                        "unit": "Mpixel/s", "gbs": (h2d + d2h) / copy_ceiling["ms"] / 1e6,
                        "what": "the same step's host-to-device and device-to-host copies "
                                "alone, same streams (the host link's ceiling for e2e)"}},
            "issue_roofline": issue,
            "per_frame_launch": per_frame,
            "schedules": {"autotuned": tuned, "ms_per_step": by_schedule,
                          "what": "each a CUDA graph of one sb_stylize_batch launch over the "
                                  "step's frames; persistent = resident CTAs taking tiles from "
                                  "a work queue; interleave_rows = tile row r of every frame "
                                  "before row r + 1"},
            "lookup_only": lookup,
            "gpu_launches": args.steps,
            "lut_build_ms": min(t_lut),
            "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_served:
        line["served"] = run_served(dev)
    if rank == 0 and world == 1 and not args.no_uneven:
        line["batched_uneven"] = run_uneven(dev)
    if rank == 0 and world == 1 and args.workload == "1080p" and not args.no_4k:
        line["workload_4k"] = run_workload_4k(dev, min(args.steps, 300), max(3, args.warmup))
    if rank == 0:
        line["workload_stats"] = workload_stats(sb, g_tgt[0], g_src, lut, w, w.blend_radius)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = cpu_oracle_run(w, frames)
        line["cpu_baseline"] = {k: r[k] for k in ("value", "unit", "cores", "kind", "sample")}
        # one core: the kind of figure the paper quotes (seconds per frame on a
        # single-core CPU), context only
        r1 = cpu_oracle_run(w, frames, budget_s=6.0, threads=1)
        line["cpu_baseline"]["single_core"] = {
            "value": r1["value"], "unit": "Mpixel/s",
            "s_per_frame": W * H / (r1["value"] * 1e6), "sample": r1["sample"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    lut.destroy()
    if world > 1:
        dist.destroy_process_group()


def copies_only(dev, host_in, host_out, staging, streams, main, reps: int = 10) -> dict:
    """Times one e2e step's copies without the kernels: every guide in and
    every output out through the staging buffers, groups over the same
    streams.  The result bounds what any e2e step can reach on this host link."""
    import torch

    bufs = list(staging.values())
    assert len(bufs) == len(host_in)

    def step():
        for g0 in range(0, len(bufs), E2E_GROUP):
            st = streams[(g0 // E2E_GROUP) % len(streams)]
            with torch.cuda.stream(st):
                for k in range(g0, min(len(bufs), g0 + E2E_GROUP)):
                    bufs[k][0].copy_(host_in[k], non_blocking=True)
                    host_out[k].copy_(bufs[k][1], non_blocking=True)

    step()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(main):
        t0.record(main)
    for st in streams:
        st.wait_event(t0)
    for _ in range(reps):
        step()
    for st in streams:
        ev = torch.cuda.Event()
        ev.record(st)
        main.wait_event(ev)
    with torch.cuda.stream(main):
        t1.record(main)
    torch.cuda.synchronize()
    return {"ms": t0.elapsed_time(t1) / reps}


def workload_stats(sb, g_tgt, g_src, lut, w, radius: int, n_sample: int = 20000,
                   seed: int = 7) -> dict:
    """Method statistics of one frame (from sb_assign_chunks): accepted-level
    histogram and mean, and over a pixel sample the mean number of distinct
    chunk translations A(n) - n in the vote window (1 = a plain copy) and the
    share of windows with more than one."""
    import torch
    A, lev = sb.assign_chunks(g_tgt, g_src, lut, w.levels, w.threshold, w.seed)
    torch.cuda.synchronize()
    a = A.cpu().numpy().astype(np.int64)
    lv = lev.cpu().numpy()
    H, W = a.shape
    hist = np.bincount(lv.ravel(), minlength=w.levels + 1)[1:]
    ys, xs = np.mgrid[0:H, 0:W]
    dx = (a & 0xFFFF) - xs
    dy = (a >> 16) - ys
    d = (dy + 65536) * 262144 + (dx + 65536)  # translation as one integer
    rng = np.random.default_rng(seed)
    px = rng.integers(0, W, n_sample)
    py = rng.integers(0, H, n_sample)
    counts = np.empty(n_sample, np.int64)
    offs = np.arange(-radius, radius + 1)
    for k in range(n_sample):
        yy = np.clip(py[k] + offs, 0, H - 1)
        xx = np.clip(px[k] + offs, 0, W - 1)
        win = d[np.ix_(np.unique(yy), np.unique(xx))]
        counts[k] = len(np.unique(win))
    # texture coherence: share of horizontally adjacent pixels whose source
    # positions are adjacent too, for StyleBlit and for the lookup-only
    # comparator (its source map read back through a style that holds each
    # texel's own coordinates)
    Hs, Ws = g_src.shape[:2]
    yy, xx = np.mgrid[0:Hs, 0:Ws]
    coord = np.stack([xx & 0xFF, xx >> 8, yy & 0xFF, yy >> 8], axis=-1).astype(np.uint8)
    lk = sb.lookup_only(g_tgt, g_src, torch.from_numpy(coord).to(g_tgt.device), lut)
    torch.cuda.synchronize()
    lkc = lk.cpu().numpy().astype(np.int64)
    lx, ly = lkc[..., 0] | (lkc[..., 1] << 8), lkc[..., 2] | (lkc[..., 3] << 8)

    def coherent(sx, sy):
        return float(((sx[:, 1:] == sx[:, :-1] + 1) & (sy[:, 1:] == sy[:, :-1])).mean())

    return {"level_histogram": {f"L{l + 1}": int(c) for l, c in enumerate(hist)},
            "mean_accepted_level": float((np.arange(1, w.levels + 1) * hist).sum() / hist.sum()),
            "source_coherence": {"stylize": coherent(a & 0xFFFF, a >> 16),
                                 "lookup_only": coherent(lx, ly)},
            "mean_distinct_translations_per_window": float(counts.mean()),
            "windows_with_several_translations": float((counts > 1).mean()),
            "sample": f"frame 0, {n_sample} pixels for the window statistics (window clipped "
                      "at frame borders)"}


def run_workload_4k(dev, steps: int, warmup: int) -> dict:
    """The 3840x2160 UV workload (L7, T 2^20, 7x7 vote, 2048^2 identity-UV
    exemplar): one sb_stylize_batch launch over FRAMES_PER_STEP distinct
    frames per step (a CUDA graph; inputs and outputs exceed L2), with its HBM
    roofline and issue roofline, and the single-frame path (one sb_stylize
    launch per frame, the same frames in turn, so no frame is L2-resident when
    its launch starts)."""
    import torch

    import paper_1807_03249_gb300 as sb
    w, frames = make_workload("4k", FRAMES_PER_STEP)
    ex = w.exemplar
    H, W = frames[0].shape[:2]
    ab = algorithmic_bytes(w, frames[0])

    def to_dev(a):
        return torch.from_numpy(np.ascontiguousarray(a.view(np.int16) if a.dtype == np.uint16
                                                     else a)).to(dev)

    gs, st = to_dev(ex.guide), to_dev(ex.style)
    lut = sb.build_lut(gs, ex.lut_bits)
    gts = [to_dev(f) for f in frames]
    outs = [torch.empty((H, W, 4), dtype=torch.uint8, device=dev) for _ in frames]
    batch = [sb.BatchFrame(gts[i], lut, st, w.levels, w.threshold, w.seed + i, out=outs[i])
             for i in range(FRAMES_PER_STEP)]
    stream = torch.cuda.Stream(dev)

    def graph_of(fn):
        with torch.cuda.stream(stream):
            fn()
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            fn()
        torch.cuda.synchronize()
        for _ in range(warmup):
            with torch.cuda.stream(stream):
                g.replay()
        torch.cuda.synchronize()
        return g

    def timed(g, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(n):
                g.replay()
            e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    def singles():
        for i in range(FRAMES_PER_STEP):
            sb.stylize(gts[i], gs, st, lut, w.levels, w.threshold, w.blend_radius, w.seed + i,
                       out=outs[i], stream=stream)

    tuned, _ = sb.autotune_batch(batch, w.blend_radius, reps=3, stream=stream)
    torch.cuda.synchronize()
    ms_batch = timed(graph_of(lambda: sb.stylize_batch(batch, w.blend_radius, stream=stream,
                                                       schedule=tuned)), steps)
    by_schedule = {}
    for rows in (32, 16, 64):
        for pers in (0, 1):
            for il in (0, 1):
                sc = {"persistent": pers, "largest_first": 0, "interleave_rows": il,
                      "tile_rows": rows}
                by_schedule[f"tile_rows={rows},persistent={pers},interleave_rows={il}"] = timed(
                    graph_of(lambda: sb.stylize_batch(batch, w.blend_radius, stream=stream,
                                                      schedule=sc)), max(10, steps // 3))
    ms_single = timed(graph_of(singles), max(3, steps // 2)) / FRAMES_PER_STEP
    lut.destroy()
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs") or 6800.0
    alg = FRAMES_PER_STEP * ab["frame_bytes"] + ab["exemplar_bytes"]
    achieved = alg / (ms_batch / 1e3) / 1e9
    counters = profiled_counters("4k", tuned)
    sm_mhz = peaks.get("sm_max_mhz") or 2070.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    issue_peak = sms * 4 * sm_mhz * 1e6
    inst = counters.get("warp_instructions_per_launch")
    single_bytes = ab["frame_bytes"] + ab["exemplar_bytes"]
    return {"workload": w.name, "frame": f"{W}x{H}", "frames_per_step": FRAMES_PER_STEP,
            "levels": w.levels, "threshold": w.threshold,
            "blend": f"{2 * w.blend_radius + 1}x{2 * w.blend_radius + 1}",
            "value": job_throughput(1, FRAMES_PER_STEP * H * W, 1, ms_batch),
            "unit": "Mpixel/s", "ms_per_step": ms_batch, "steps": steps,
            "schedule": tuned, "ms_per_step_by_schedule": by_schedule,
            "us_per_frame": 1e3 * ms_batch / FRAMES_PER_STEP,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm,
                         "traffic": counters.get("dram_bytes_per_launch"),
                         "kernel": f"batch_kernel{'_persistent' if tuned.get('persistent') else ''}"
                                   f"<2,16,{w.blend_radius},{int(tuned.get('tile_rows') or 32)}> "
                                   f"(sb_stylize_batch)",
                         "algorithmic_bytes_per_launch": alg,
                         "bytes_rule": "24 frames x (guide in + RGBA8 out) + exemplar "
                                       "(style + guide + table) once per launch"},
            "issue_roofline": {"bound": "issue", "unit": "warp instructions/s",
                               "peak": issue_peak,
                               "achieved": inst / (ms_batch / 1e3) if inst else None,
                               "frac": inst / (ms_batch / 1e3) / issue_peak if inst else None,
                               "instructions_per_launch": inst},
            "single_frame": {"us_per_frame": 1e3 * ms_single,
                             "value": H * W / (ms_single / 1e3) / 1e6, "unit": "Mpixel/s",
                             "hbm_frac": single_bytes / (ms_single / 1e3) / 1e9 / hbm,
                             "bytes_rule": "guide in + RGBA8 out + exemplar (style + guide + "
                                           "table) per frame",
                             "launch": "CUDA graph of 24 sb_stylize launches, one per frame"}}


def run_uneven(dev, n_frames: int = 64, n_exemplars: int = 8, seed: int = 4000,
               steps: int = 20) -> dict:
    """The uneven batch: n_frames frames with widths uniform in [640, 3840]
    (16:9), each stylised with one of n_exemplars 1024^2 sphere-guide
    exemplars, L=6, T=300, 5x5 blend.  Frames are crops of two generated
    3840x2160 normal fields.  Times per step: one sb_stylize per frame (a CUDA
    graph of n_frames launches), one default batch launch, and the batch launch
    under the schedule sb_autotune_batch picks (each a CUDA graph); checks that
    the three give the same pixels."""
    import torch

    import paper_1807_03249_gb300 as sb
    exs = []
    for k in range(n_exemplars):
        ex = synth.normal_exemplar(seed + 100 + k, 1024, strokes=100, octaves=3, lut_bits=6)
        gs, st = torch.from_numpy(ex.guide).to(dev), torch.from_numpy(ex.style).to(dev)
        exs.append((gs, st, sb.build_lut(gs, ex.lut_bits)))
    fields = [synth.bump_normals(seed + k, 2160, 3840, 64, (20.0, 200.0)) for k in range(2)]
    sizes = synth.batch_frame_sizes(seed, n_frames)
    rng = np.random.default_rng(seed + 1)
    frames, singles = [], []
    for i, (w_, h_) in enumerate(sizes):
        f = fields[i % 2]
        y0, x0 = int(rng.integers(0, 2160 - h_ + 1)), int(rng.integers(0, 3840 - w_ + 1))
        g = torch.from_numpy(np.ascontiguousarray(f[y0:y0 + h_, x0:x0 + w_])).to(dev)
        gs, st, lut = exs[int(rng.integers(0, n_exemplars))]
        sd = int(rng.integers(0, 2**32))
        frames.append(sb.BatchFrame(g, lut, st, 6, 300, sd))
        singles.append((g, gs, st, lut, sd, torch.empty_like(frames[-1].out)))
    px = sum(f.tgt_guide.shape[0] * f.tgt_guide.shape[1] for f in frames)
    stream = torch.cuda.Stream(dev)

    def per_frame():
        for g, gs, st, lut, sd, o in singles:
            sb.stylize(g, gs, st, lut, 6, 300, 2, sd, out=o)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            fn()
        for _ in range(3):
            graph.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with torch.cuda.stream(stream):
            for _ in range(steps):
                graph.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    ms_pf = timed(per_frame)
    ms_batch = timed(lambda: sb.stylize_batch(frames, 2))
    best, _ = sb.autotune_batch(frames, 2, reps=3)
    ms_tuned = timed(lambda: sb.stylize_batch(frames, 2, schedule=best))
    per_schedule = {}
    for rows in (32, 16, 64):
        for pers in (0, 1):
            for lf in (0, 1):
                sc = {"persistent": pers, "largest_first": lf, "tile_rows": rows}
                per_schedule[f"tile_rows={rows},persistent={pers},largest_first={lf}"] = timed(
                    lambda: sb.stylize_batch(frames, 2, schedule=sc))
    torch.cuda.synchronize()
    equal = all(torch.equal(f.out, o) for f, (_, _, _, _, _, o) in zip(frames, singles))
    for _, _, lut in exs:
        lut.destroy()
    return {"frames": n_frames, "exemplars": n_exemplars, "mpixel_per_step": px / 1e6,
            "per_frame_launch_frames_per_s": n_frames / (ms_pf / 1e3),
            "batch_frames_per_s": n_frames / (ms_batch / 1e3),
            "autotuned_frames_per_s": n_frames / (ms_tuned / 1e3),
            "autotuned_mpixel_per_s": px / (ms_tuned / 1e3) / 1e6,
            "autotuned_schedule": best, "equal_outputs": equal,
            "ms_per_step": {"per_frame": ms_pf, "batch": ms_batch, "autotuned": ms_tuned},
            "ms_per_step_by_schedule": per_schedule,
            "workload": f"{n_frames} frames 640x360..3840x2160 (16:9), {n_exemplars} 1024^2 "
                        "sphere exemplars, L6 T300 5x5; each form a CUDA graph"}


def run_served(dev, n_requests: int = 10000, rate_hz: float = 2000.0, pool: int = 64,
               seed: int = 5000) -> dict:
    """The served workload: a seeded Poisson stream of stylisation requests,
    frame sizes log-uniform in [256^2, 3840x2160], 16 resident 1024^2
    exemplars, 40 GB admission budget, 5x5 blend, L=6, T=300, served three
    times (each pass's p50/p99 and longest host-loop gap are reported; the
    headline is the pass with the median p99).  Request guides
    are crops of one generated 3840x2160 normal field held in a pool of pinned
    buffers (outputs of the same pool entry are overwritten; they are not
    checked here -- tests/test_gpu_serve.py checks served results)."""
    import torch

    from paper_1807_03249_gb300.serve import Request, Server, latency_summary
    srv = Server(dev, radius=2, budget_bytes=40 << 30, slots=4, max_batch=16)
    for k in range(16):
        ex = synth.normal_exemplar(5100 + k, 1024, strokes=100, lut_bits=6)
        srv.add_exemplar(k, ex.guide, ex.style, ex.lut_bits)
    field = synth.bump_normals(seed, 2160, 3840, 96, (20.0, 200.0))
    sizes = synth.log_uniform_sizes(seed + 1, pool)
    rng = np.random.default_rng(seed + 2)
    guides, outs = [], []
    for (w_, h_) in sizes:
        y0, x0 = int(rng.integers(0, 2160 - h_ + 1)), int(rng.integers(0, 3840 - w_ + 1))
        guides.append(torch.from_numpy(np.ascontiguousarray(field[y0:y0 + h_, x0:x0 + w_]))
                      .pin_memory())
        outs.append(torch.empty((h_, w_, 4), dtype=torch.uint8).pin_memory())
    arrivals = synth.poisson_arrivals(seed + 3, rate_hz, n_requests)
    exs = rng.integers(0, 16, n_requests)
    seeds = rng.integers(0, 2**32, n_requests)

    def make(i, t0):
        return Request(i, float(arrivals[i] - t0), int(exs[i]), guides[i % pool], 6, 300,
                       int(seeds[i]), out=outs[i % pool])

    # slot arenas sized for the largest possible group before anything is timed
    srv.reserve(sum(sorted(srv.device_bytes(g) for g in guides)[-srv.sched.max_batch:]))
    warm = [make(i, arrivals[0]) for i in range(64)]
    srv.run(warm, real_time=False)
    # three independent passes over the same arrival stream; the headline is
    # the pass with the median p99 (a single host stall moves one pass's p99)
    runs = []
    for _ in range(3):
        reqs = [make(i, arrivals[0]) for i in range(n_requests)]
        done, wall = srv.run(reqs, real_time=True)
        r = latency_summary(done, wall)
        r["max_loop_gap_ms"] = srv.max_loop_gap_s * 1e3
        runs.append(r)
    out = dict(sorted(runs, key=lambda r: r["p99_ms"])[1])
    out["runs"] = [{k: r[k] for k in ("p50_ms", "p99_ms", "mean_ms", "max_loop_gap_ms")}
                   for r in runs]

    # saturation: the same kind of requests all waiting at once, served by the
    # continuous-batching loop vs one plain sb_stylize per request (with the
    # same copies) on one stream
    import paper_1807_03249_gb300 as sb
    n_sat = min(2000, n_requests)
    sat = [make(i, arrivals[0]) for i in range(n_sat)]
    _, wall_sat = srv.run(sat, real_time=False)
    px_sat = sum(r.pixels for r in sat)
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for r in sat:
            g = torch.empty(r.guide.shape, dtype=r.guide.dtype, device=dev)
            g.copy_(r.guide, non_blocking=True)
            gd, sd, lut = srv.exemplars[r.exemplar]
            o = sb.stylize(g, gd, sd, lut, r.levels, r.threshold, 2, r.seed, stream=stream)
            r.out.copy_(o, non_blocking=True)
    torch.cuda.synchronize()
    wall_seq = time.perf_counter() - t0
    out["saturated"] = {"requests": n_sat,
                        "batched_frames_per_s": n_sat / wall_sat,
                        "batched_mpixel_per_s": px_sat / wall_sat / 1e6,
                        "per_request_frames_per_s": n_sat / wall_seq,
                        "per_request_mpixel_per_s": px_sat / wall_seq / 1e6,
                        "what": "all requests waiting at t=0: serving loop (4 slots, groups of "
                                "<= 16) vs one sb_stylize per request on one stream"}
    offered_px = sum(r.pixels for r in reqs) / float(arrivals[-1] - arrivals[0])
    out.update({"offered_req_per_s": rate_hz, "offered_mpixel_per_s": offered_px / 1e6,
                "slots": 4, "max_batch": 16, "budget_gb": 40,
                "peak_admitted_mb": srv.sched.peak_in_use / 1e6,
                "workload": "Poisson 2000 req/s, log-uniform 256^2..3840x2160 normals, "
                            "16 resident 1024^2 exemplars, L6 T300 5x5"})
    return out


def profile_once(args):
    import torch

    import paper_1807_03249_gb300 as sb
    dev = torch.device("cuda:0")
    w, frames = make_workload(args.workload, FRAMES_PER_STEP)
    ex = w.exemplar

    def to_dev(a):
        return torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).to(dev)

    gs, st = to_dev(ex.guide), to_dev(ex.style)
    lut = sb.build_lut(gs, ex.lut_bits)
    batch = [sb.BatchFrame(to_dev(f), lut, st, w.levels, w.threshold, w.seed + i)
             for i, f in enumerate(frames)]
    pers, lf, il, rows = (int(v) for v in args.schedule.split(","))
    sched = {"persistent": pers, "largest_first": lf, "interleave_rows": il, "tile_rows": rows}
    for _ in range(2):
        sb.stylize_batch(batch, w.blend_radius, schedule=sched)
    # then, if asked, the single-frame path: one sb_stylize per frame
    for i in range(min(args.single_frames, len(batch))):
        f = batch[i]
        sb.stylize(f.tgt_guide, gs, st, lut, w.levels, w.threshold, w.blend_radius, f.seed,
                   out=f.out)
    # then the lookup-only comparator over the same frames, batched, twice
    for _ in range(2):
        sb.lookup_only_batch(batch)
    torch.cuda.synchronize()
    print(json.dumps({"profile_once": w.name, "frames": len(batch), "schedule": sched,
                      "single_frames": min(args.single_frames, len(batch))}))


def main():
    args = _args()
    if args.profile_once:
        profile_once(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

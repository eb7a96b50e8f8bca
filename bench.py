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
    return p.parse_args()


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def make_workload(name: str, n_frames: int, rank: int = 0):
    """Exemplar + `n_frames` distinct target guides (a few generated fields,
    each shifted cyclically by seeded offsets)."""
    base = 3 if name == "1080p" else 2
    seed0 = (2000 if name == "1080p" else 3000) + 100 * rank
    w = synth.workload_1080p(base, seed0) if name == "1080p" else synth.workload_4k_uv(base, seed0)
    rng = np.random.default_rng(seed0)
    frames = []
    for i in range(n_frames):
        g = w.frames[i % base].guide
        dy, dx = int(rng.integers(0, g.shape[0])), int(rng.integers(0, g.shape[1]))
        frames.append(np.ascontiguousarray(np.roll(g, (dy, dx), axis=(0, 1))))
    return w, frames


def algorithmic_bytes(w, frame) -> dict:
    H, W, C = frame.shape
    px = H * W
    guide_b = px * C * frame.dtype.itemsize
    out_b = px * 4
    ex = w.exemplar
    ex_b = ex.style.nbytes + ex.guide.nbytes + 4 * (1 << (ex.guide.shape[2] * ex.lut_bits))
    return dict(pixels=px, frame_bytes=guide_b + out_b, exemplar_bytes=ex_b)


def kernel_source_hash() -> str:
    d = os.path.join(ROOT, "paper_1807_03249_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh")):
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", f"sb_stylize_batch_{workload}_traffic.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_source_hash") != kernel_source_hash():
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


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

def cpu_oracle_run(w, frames, budget_s: float = 12.0, steps: int | None = None):
    """Times the oracle (assignment + RGBA8 vote) on a band of rows of the
    workload's frames with every host core; look-up table entries the band
    needs are filled in an untimed pass first (the GPU also runs with a
    resident table)."""
    import oracle
    ex = w.exemplar
    cores = os.cpu_count() or 1
    lut = oracle.new_lut(ex.guide.shape[2], ex.lut_bits)
    rows = 64
    band = [np.ascontiguousarray(f[:rows]) for f in frames[:2]]
    for i, g in enumerate(band):  # untimed: fill the table entries the band needs
        oracle.assign(g, ex.guide, ex.lut_bits, w.levels, w.threshold, w.seed + i, lut=lut,
                      n_threads=cores)
    times, px = [], 0
    t_start = time.perf_counter()
    n = 0
    while True:
        g = band[n % len(band)]
        t = time.perf_counter()
        a, _ = oracle.assign(g, ex.guide, ex.lut_bits, w.levels, w.threshold, w.seed + n % 2,
                             lut=lut, n_threads=cores)
        oracle.blend_rgba8(a, ex.style, w.blend_radius, n_threads=cores)
        times.append(time.perf_counter() - t)
        px += g.shape[0] * g.shape[1]
        n += 1
        if steps is not None and n >= steps:
            break
        if steps is None and time.perf_counter() - t_start > budget_s:
            break
    total = sum(times)
    return {"value": px / total / 1e6, "unit": "Mpixel/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} x {rows}-row bands ({rows}x{band[0].shape[1]} px) of the "
                      f"{w.name} frames, assignment + r={w.blend_radius} vote, "
                      f"table entries filled in an untimed pass",
            "seconds": total}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w, frames = make_workload(args.workload, 2)
    r = cpu_oracle_run(w, frames, steps=None, budget_s=max(5.0, min(60.0, 0.5 * args.steps)))
    H, W = frames[0].shape[:2]
    line = {"metric": METRIC, "value": r["value"], "unit": "Mpixel/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": w.name, "frame": f"{W}x{H}", "levels": w.levels,
                       "threshold": w.threshold, "blend": f"{2 * w.blend_radius + 1}x"
                       f"{2 * w.blend_radius + 1}"},
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

    def step_batch():
        sb.stylize_batch(batch, w.blend_radius, stream=stream)

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
        t = e0.elapsed_time(e1)
        if world > 1:
            tt = torch.tensor([t], device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            t = float(tt.item())
        return t

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
    value = world * px_step * args.steps / (ms / 1e3) / 1e6
    pf_steps = max(3, min(args.steps, 300))
    ms_pf = time_graph(graph_frames, pf_steps)
    per_frame = {"value": world * px_step * pf_steps / (ms_pf / 1e3) / 1e6, "unit": "Mpixel/s",
                 "ms_per_step": ms_pf / pf_steps, "steps": pf_steps,
                 "launch": "CUDA graph of frames_per_step sb_stylize kernels (one per frame)"}

    # end to end through the host-buffer call: pinned H2D, stylise, D2H, with
    # frames spread over three streams so copies in both directions overlap
    host_in = [torch.from_numpy(f.view(np.int16) if f.dtype == np.uint16 else f).pin_memory()
               for f in frames]
    host_out = [torch.empty((H, W, 4), dtype=torch.uint8).pin_memory() for _ in frames]
    staging = [dict() for _ in frames]
    e2e_streams = [torch.cuda.Stream(dev) for _ in range(3)]

    def e2e_step():
        for i in range(FRAMES_PER_STEP):
            sb.stylize_host(host_in[i], g_src, style, lut, w.levels, w.threshold,
                            w.blend_radius, w.seed + i, host_out[i], staging=staging[i],
                            stream=e2e_streams[i % 3])

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
    ms_e2e = x0.elapsed_time(x1)
    if world > 1:
        t = torch.tensor([ms_e2e], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_e2e = float(t.item())
    e2e_value = world * px_step * args.e2e_steps / (ms_e2e / 1e3) / 1e6
    h2d = sum(f.nbytes for f in frames)
    d2h = sum(o.numel() for o in host_out)

    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    kernel_s = ms_per_step / 1e3  # one batch launch per step
    alg = FRAMES_PER_STEP * ab["frame_bytes"] + ab["exemplar_bytes"]
    achieved = alg / kernel_s / 1e9
    traffic = profiled_traffic(args.workload)

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
                                 "frames_per_step frames",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic,
                         "kernel": "batch_kernel<3,8,2> (sb_stylize_batch)",
                         "peak_source": f"{peak_src} copy bandwidth",
                         "algorithmic_bytes_per_launch": alg,
                         "frame_only_frac": FRAMES_PER_STEP * ab["frame_bytes"] / kernel_s
                         / 1e9 / hbm,
                         "kernel_us": kernel_s * 1e6,
                         "bytes_rule": "24 frames x (guide in + RGBA8 out) + exemplar "
                                       "(style + guide + table) once per launch"},
            "e2e": {"value": e2e_value, "unit": "Mpixel/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
                    "api": "stylize_host per frame (pinned host in/out), 3 streams"},
            "per_frame_launch": per_frame,
            "gpu_launches": args.steps,
            "lut_build_ms": min(t_lut),
            "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = cpu_oracle_run(w, frames)
        line["cpu_baseline"] = {k: r[k] for k in ("value", "unit", "cores", "kind", "sample")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    lut.destroy()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

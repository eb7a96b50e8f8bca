"""The multi-rank host logic of bench.py on CPU with the gloo backend
(world size 2): ranks stylise disjoint frames, the job time is the slowest
rank's, and throughput counts every rank's pixels.  No GPU is involved."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import synth
        seed = bench.rank_frame_seed("1080p", rank)
        # this rank's frames: a small field from the same generator and seed rule
        g = synth.bump_normals(seed, 36, 64, 4, (5.0, 20.0))
        ms = [3.0, 5.0][rank]
        worst = bench.max_over_ranks(ms, world)
        value = bench.job_throughput(world, 1000, 10, worst)
        q.put((rank, seed, g.tobytes(), worst, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_frames_and_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    (r0, s0, g0, w0, v0), (r1, s1, g1, w1, v1) = out
    assert s0 != s1 and g0 != g1          # disjoint frames per rank
    assert w0 == w1 == 5.0                # both ranks report the slowest time
    assert v0 == v1 == pytest.approx(2 * 1000 * 10 / 5e-3 / 1e6)

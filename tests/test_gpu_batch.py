"""sb_stylize_batch: many frames of mixed sizes, exemplars, levels, thresholds
and seeds in one launch must give, frame by frame, exactly what sb_stylize
gives for that frame alone, and what the oracle gives."""
import os

import numpy as np
import pytest
import torch

import oracle
import paper_1807_03249_gb300 as sb
import synth
from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu


def _exemplars(dev, n):
    out = []
    for k in range(n):
        size = [64, 96, 128][k % 3]
        g = synth.sphere_normals(size)
        st = synth.value_noise_style(70 + k, size, size, octaves=3, base_cell=16)
        gd, sd = to_dev(g, dev), to_dev(st, dev)
        out.append((g, st, gd, sd, sb.build_lut(gd, 5)))
    return out


@pytest.mark.parametrize("radius", [0, 2, 3])
def test_batch_equals_single_frame_calls(cuda_device, radius):
    rng = np.random.default_rng(radius)
    exs = _exemplars(cuda_device, 3)
    frames, singles, hosts = [], [], []
    for k in range(9):
        W, H = int(rng.integers(1, 300)), int(rng.integers(1, 200))
        if k == 4:
            W, H = 0, 17  # empty frame inside the batch
        g = synth.bump_normals(900 + k, H, W, 3, (6.0, 40.0)) if W * H else \
            np.zeros((H, W, 3), np.uint8)
        e = exs[k % 3]
        levels, T, seed = int(rng.integers(1, 7)), int(rng.integers(0, 2000)), int(rng.integers(0, 2**32))
        gd = to_dev(g, cuda_device)
        frames.append(sb.BatchFrame(gd, e[4], e[3], levels, T, seed))
        singles.append(sb.stylize(gd, e[2], e[3], e[4], levels, T, radius, seed))
        hosts.append((g, e, levels, T, seed))
    outs = sb.stylize_batch(frames, radius)
    torch.cuda.synchronize()
    for k, (o, s1) in enumerate(zip(outs, singles)):
        assert torch.equal(o, s1), f"frame {k}"
    # two frames against the oracle, whole frame
    for k in (0, 5):
        g, e, levels, T, seed = hosts[k]
        ref, _, _ = oracle.stylize(g, e[0], e[1], 5, levels, T, radius, seed)
        assert np.array_equal(outs[k].cpu().numpy(), ref)


def test_batch_full_size_frames_persistent_whole_frames(cuda_device):
    """Full-size 1080p frames through the persistent work-queue schedule,
    largest frames first: every pixel equals the oracle."""
    w = synth.workload_1080p(2)
    ex = w.exemplar
    gs, st = to_dev(ex.guide, cuda_device), to_dev(ex.style, cuda_device)
    lut = sb.build_lut(gs, ex.lut_bits)
    frames = [sb.BatchFrame(to_dev(f.guide, cuda_device), lut, st, w.levels, w.threshold,
                            w.seed + i) for i, f in enumerate(w.frames)]
    outs = sb.stylize_batch(frames, w.blend_radius,
                            schedule={"persistent": 1, "largest_first": 1})
    torch.cuda.synchronize()
    ref_lut = oracle.new_lut(ex.guide.shape[2], ex.lut_bits)
    for i, f in enumerate(w.frames):
        ref, _, _ = oracle.stylize(f.guide, ex.guide, ex.style, ex.lut_bits, w.levels,
                                   w.threshold, w.blend_radius, w.seed + i, lut=ref_lut,
                                   n_threads=os.cpu_count() or 1)
        assert np.array_equal(outs[i].cpu().numpy(), ref), f"frame {i}"


def test_batch_argument_errors(cuda_device):
    exs = _exemplars(cuda_device, 1)
    g8 = to_dev(synth.random_guide(1, 20, 20, 3), cuda_device)
    g2 = to_dev(synth.random_guide(2, 20, 20, 2), cuda_device)
    f_ok = sb.BatchFrame(g8, exs[0][4], exs[0][3], 3, 100, 1)
    assert sb.stylize_batch([], 2) == []
    with pytest.raises(sb.StyleBlitError):
        sb.stylize_batch([f_ok], 16)                                  # radius above 15
    with pytest.raises(sb.StyleBlitError):
        sb.stylize_batch([sb.BatchFrame(g8, exs[0][4], exs[0][3], 16, 1, 1)], 1)  # levels above 15
    with pytest.raises(sb.StyleBlitError) as e:
        sb.stylize_batch([f_ok, sb.BatchFrame(g2, exs[0][4], exs[0][3], 3, 1, 1)], 1)
    assert e.value.status in (-1, -2)
    with pytest.raises(sb.StyleBlitError):
        sb.stylize_batch([f_ok] * (sb.MAX_BATCH + 1), 1)
    torch.cuda.synchronize()


@pytest.mark.parametrize("group,n_streams", [(2, 2), (3, 1), (7, 3)])
def test_host_buffer_calls_equal_device_calls(cuda_device, group, n_streams):
    """stylize_host and stylize_batch_host (pinned host in and out, copies and
    launches on the given streams) give the device calls' pixels."""
    exs = _exemplars(cuda_device, 2)
    rng = np.random.default_rng(group)
    guides, luts, styles, levels, Ts, seeds = [], [], [], [], [], []
    for k in range(7):
        W, H = int(rng.integers(30, 250)), int(rng.integers(20, 150))
        guides.append(synth.bump_normals(500 + k, H, W, 3, (6.0, 40.0)))
        e = exs[k % 2]
        luts.append(e[4])
        styles.append(e[3])
        levels.append(int(rng.integers(1, 7)))
        Ts.append(int(rng.integers(0, 2000)))
        seeds.append(int(rng.integers(0, 2**32)))
    host_in = [torch.from_numpy(g).pin_memory() for g in guides]
    host_out = [torch.empty((g.shape[0], g.shape[1], 4), dtype=torch.uint8).pin_memory()
                for g in guides]
    streams = [torch.cuda.Stream(cuda_device) for _ in range(n_streams)]
    sb.stylize_batch_host(host_in, luts, styles, levels, Ts, seeds, 2, host_out, group=group,
                          streams=streams)
    torch.cuda.synchronize()
    single_out = [torch.empty_like(o).pin_memory() for o in host_out]
    for k in range(7):
        sb.stylize_host(host_in[k], exs[k % 2][2], styles[k], luts[k], levels[k], Ts[k], 2,
                        seeds[k], single_out[k], stream=streams[k % n_streams])
    torch.cuda.synchronize()
    for k in range(7):
        ref = sb.stylize(to_dev(guides[k], cuda_device), exs[k % 2][2], styles[k], luts[k],
                         levels[k], Ts[k], 2, seeds[k]).cpu()
        assert torch.equal(host_out[k], ref), f"frame {k}"
        assert torch.equal(single_out[k], ref), f"frame {k}"


def _uneven_batch(dev, n, seed):
    """Frames of mixed sizes (some empty-ish and tiny), exemplars, levels
    (1 and above 8 included), thresholds and seeds."""
    rng = np.random.default_rng(seed)
    exs = _exemplars(dev, 3)
    frames = []
    for k in range(n):
        W, H = int(rng.integers(1, 700)), int(rng.integers(1, 400))
        g = synth.bump_normals(1300 + k, H, W, 3, (6.0, 40.0))
        e = exs[k % 3]
        levels = [1, 9, 12][k % 3] if k < 3 else int(rng.integers(2, 8))
        frames.append(sb.BatchFrame(to_dev(g, dev), e[4], e[3], levels,
                                    int(rng.integers(0, 3000)), int(rng.integers(0, 2**32))))
    return frames


@pytest.mark.parametrize("radius", [1, 2, 3])
def test_every_schedule_gives_the_same_pixels(cuda_device, radius):
    """One CTA per tile or a persistent work queue, frame order or largest
    frames first: bit-identical outputs."""
    frames = _uneven_batch(cuda_device, 11, radius)
    ref = [o.clone() for o in sb.stylize_batch(frames, radius)]
    for rows in (32, 16, 64):
        for persistent in (0, 1):
            for largest_first in (0, 1):
                for f in frames:
                    f.out.zero_()
                outs = sb.stylize_batch(frames, radius,
                                        schedule={"persistent": persistent,
                                                  "largest_first": largest_first,
                                                  "interleave_rows": 1,  # mixed grids: frame order
                                                  "tile_rows": rows})
                torch.cuda.synchronize()
                for k, (o, r) in enumerate(zip(outs, ref)):
                    assert torch.equal(o, r), f"schedule {rows}/{persistent}{largest_first} frame {k}"


@pytest.mark.parametrize("radius", [2, 3])
def test_interleaved_tile_rows_give_the_same_pixels(cuda_device, radius):
    """Frames sharing one tile grid (different sizes inside the same 64 x 32
    tiling, exemplars, levels and seeds) with their tile rows interleaved,
    one CTA per tile and persistent: every frame equals the frame-order
    launch and the oracle."""
    rng = np.random.default_rng(60 + radius)
    exs = _exemplars(cuda_device, 3)
    frames, hosts = [], []
    for k in range(6):
        W, H = 256 - int(rng.integers(0, 60)), 150 - int(rng.integers(0, 20))  # 4 x 5 tiles each
        g = synth.bump_normals(1500 + k, H, W, 3, (6.0, 40.0))
        e = exs[k % 3]
        levels, T, seed = int(rng.integers(2, 8)), int(rng.integers(50, 2000)), int(rng.integers(0, 2**32))
        frames.append(sb.BatchFrame(to_dev(g, cuda_device), e[4], e[3], levels, T, seed))
        hosts.append((g, e, levels, T, seed))
    ref = [o.clone() for o in sb.stylize_batch(frames, radius)]
    for rows in (32, 16, 64):
        for persistent in (0, 1):
            for f in frames:
                f.out.zero_()
            outs = sb.stylize_batch(frames, radius, schedule={"persistent": persistent,
                                                              "interleave_rows": 1,
                                                              "tile_rows": rows})
            torch.cuda.synchronize()
            assert all(torch.equal(o, r) for o, r in zip(outs, ref)), f"{rows} rows, persistent={persistent}"
    for k in (0, 3):
        g, e, levels, T, seed = hosts[k]
        want, _, _ = oracle.stylize(g, e[0], e[1], 5, levels, T, radius, seed)
        assert np.array_equal(ref[k].cpu().numpy(), want)
    best, _ = sb.autotune_batch(frames, radius, reps=1)
    assert set(best) == {"persistent", "largest_first", "interleave_rows", "tile_rows"}
    assert best["tile_rows"] in (16, 32, 64)


def test_persistent_queue_resets_across_launches_and_graph_replays(cuda_device):
    """The work queue clears itself at the end of each launch: more launches
    than queue slots, and a captured graph replayed several times, still
    cover every tile."""
    frames = _uneven_batch(cuda_device, 6, 7)
    ref = [o.clone() for o in sb.stylize_batch(frames, 2)]
    sched = {"persistent": 1, "largest_first": 1}
    for _ in range(70):  # many launches on one stream reuse its queue
        sb.stylize_batch(frames, 2, schedule=sched)
    torch.cuda.synchronize()
    assert all(torch.equal(o, r) for o, r in zip([f.out for f in frames], ref))
    stream = torch.cuda.Stream(cuda_device)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        sb.stylize_batch(frames, 2, schedule=sched)
    for _ in range(3):
        for f in frames:
            f.out.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert all(torch.equal(f.out, r) for f, r in zip(frames, ref))


def test_persistent_launches_on_unordered_streams_and_a_graph_never_share_a_queue(cuda_device):
    """Persistent batches with radius 1 and radius 2 on four streams that do
    not wait for each other (25 launches per stream, 100 in all), while a
    captured persistent batch is replayed on a fifth stream: every launch
    writes its own outputs and every output equals the one-CTA-per-tile
    schedule's."""
    sched = {"persistent": 1, "largest_first": 0}
    inputs = {r: _uneven_batch(cuda_device, 2, 40 + r) for r in (1, 2)}
    ref = {r: [o.clone() for o in sb.stylize_batch(inputs[r], r)] for r in (1, 2)}
    streams = [torch.cuda.Stream(cuda_device) for _ in range(5)]
    gframes = [sb.BatchFrame(f.tgt_guide, f.lut, f.style, f.levels, f.threshold, f.seed)
               for f in inputs[2]]
    with torch.cuda.stream(streams[4]):
        sb.stylize_batch(gframes, 2, stream=streams[4], schedule=sched)  # set-up outside capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=streams[4]):
        sb.stylize_batch(gframes, 2, stream=streams[4], schedule=sched)
    torch.cuda.synchronize()
    launches = []
    for j in range(25):
        for k, st in enumerate(streams[:4]):
            r = 1 + k % 2
            fr = [sb.BatchFrame(f.tgt_guide, f.lut, f.style, f.levels, f.threshold, f.seed)
                  for f in inputs[r]]
            with torch.cuda.stream(st):
                sb.stylize_batch(fr, r, stream=st, schedule=sched)
            launches.append((r, fr))
        if j % 5 == 0:
            with torch.cuda.stream(streams[4]):
                for f in gframes:
                    f.out.zero_()
                graph.replay()
    torch.cuda.synchronize()
    for i, (r, fr) in enumerate(launches):
        assert all(torch.equal(f.out, o) for f, o in zip(fr, ref[r])), f"launch {i} (r={r})"
    assert all(torch.equal(f.out, o) for f, o in zip(gframes, ref[2]))


def test_autotune_picks_a_schedule_and_keeps_the_pixels(cuda_device):
    frames = _uneven_batch(cuda_device, 8, 3)
    ref = [o.clone() for o in sb.stylize_batch(frames, 2)]
    best, ms = sb.autotune_batch(frames, 2, reps=2)
    torch.cuda.synchronize()
    assert best["persistent"] in (0, 1) and best["largest_first"] in (0, 1) and ms > 0
    assert all(torch.equal(f.out, r) for f, r in zip(frames, ref))
    with pytest.raises(sb.StyleBlitError):
        sb.autotune_batch(frames, 2, reps=0)


def test_every_schedule_gives_the_same_pixels_uv16(cuda_device):
    """The same for 16-bit two-channel UV guides (the 4K format), 7x7 blend."""
    src = synth.identity_uv_guide(96, 128)
    style = synth.random_style(31, 96, 128)
    gs, st = to_dev(src, cuda_device), to_dev(style, cuda_device)
    lut = sb.build_lut(gs, 8)
    rng = np.random.default_rng(5)
    frames = []
    for k in range(7):
        W, H = int(rng.integers(40, 400)), int(rng.integers(30, 260))
        g = synth.warped_uv_guide(600 + k, H, W, 96, 128, 8)
        frames.append(sb.BatchFrame(to_dev(g, cuda_device), lut, st, int(rng.integers(2, 8)),
                                    int(rng.integers(0, 1 << 21)), int(rng.integers(0, 2**32))))
    ref = [o.clone() for o in sb.stylize_batch(frames, 3)]
    for rows in (32, 16, 64):
        for persistent in (0, 1):
            for largest_first in (0, 1):
                for f in frames:
                    f.out.zero_()
                sb.stylize_batch(frames, 3, schedule={"persistent": persistent,
                                                      "largest_first": largest_first,
                                                      "tile_rows": rows})
                torch.cuda.synchronize()
                assert all(torch.equal(f.out, r) for f, r in zip(frames, ref)), (rows, persistent)
    # and one frame against the oracle
    f0 = frames[0]
    g0 = f0.tgt_guide.cpu().numpy().view(np.uint16)
    out, _, _ = oracle.stylize(g0, src, style, 8, f0.levels, f0.threshold, 3, f0.seed)
    assert np.array_equal(ref[0].cpu().numpy(), out)

"""sb_stylize_batch: many frames of mixed sizes, exemplars, levels, thresholds
and seeds in one launch must give, frame by frame, exactly what sb_stylize
gives for that frame alone (and, sampled, what the oracle gives)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1807_03249_gb300 as sb
import synth
from tests.gpu_helpers import sample_pixels, to_dev

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


def test_batch_full_size_frames_sampled(cuda_device):
    w = synth.workload_1080p(2)
    ex = w.exemplar
    gs, st = to_dev(ex.guide, cuda_device), to_dev(ex.style, cuda_device)
    lut = sb.build_lut(gs, ex.lut_bits)
    frames = [sb.BatchFrame(to_dev(f.guide, cuda_device), lut, st, w.levels, w.threshold,
                            w.seed + i) for i, f in enumerate(w.frames)]
    outs = sb.stylize_batch(frames, w.blend_radius)
    torch.cuda.synchronize()
    for i, f in enumerate(w.frames):
        xs, ys = sample_pixels(40 + i, 1920, 1080, 40, w.blend_radius)
        ref = oracle.stylize_points(f.guide, ex.guide, ex.style, ex.lut_bits, w.levels,
                                    w.threshold, w.blend_radius, w.seed + i, xs, ys)
        assert np.array_equal(outs[i].cpu().numpy()[ys, xs], ref)


def test_batch_argument_errors(cuda_device):
    exs = _exemplars(cuda_device, 1)
    g8 = to_dev(synth.random_guide(1, 20, 20, 3), cuda_device)
    g2 = to_dev(synth.random_guide(2, 20, 20, 2), cuda_device)
    f_ok = sb.BatchFrame(g8, exs[0][4], exs[0][3], 3, 100, 1)
    assert sb.stylize_batch([], 2) == []
    with pytest.raises(sb.StyleBlitError):
        sb.stylize_batch([f_ok], 8)                                   # radius
    with pytest.raises(sb.StyleBlitError):
        sb.stylize_batch([sb.BatchFrame(g8, exs[0][4], exs[0][3], 13, 1, 1)], 1)  # levels
    with pytest.raises(sb.StyleBlitError) as e:
        sb.stylize_batch([f_ok, sb.BatchFrame(g2, exs[0][4], exs[0][3], 3, 1, 1)], 1)
    assert e.value.status in (-1, -2)
    with pytest.raises(sb.StyleBlitError):
        sb.stylize_batch([f_ok] * (sb.MAX_BATCH + 1), 1)
    torch.cuda.synchronize()

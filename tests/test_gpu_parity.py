"""Parity of the CUDA library (through its C ABI) with the CPU oracle.

The bar is bit-exactness: look-up tables, assignment maps, level maps and
RGBA8 outputs are integer results and must equal the oracle's element by
element; the float vote must be within 1e-5 absolute.  Every case compares
whole frames, the 1920x1080 and 3840x2160 workloads included (several frames
in one batched launch, as the benchmark runs them).
"""
import os

import numpy as np
import pytest
import torch

import oracle
import paper_1807_03249_gb300 as sb
import synth
from tests.gpu_helpers import sample_pixels, to_dev, u32, workload
from tests.golden.cases import REGRESSION_CASES, make_case

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5


def _full(dev, c, radius=None):
    radius = c["radius"] if radius is None else radius
    gt, gs, st = to_dev(c["tgt"], dev), to_dev(c["src"], dev), to_dev(c["style"], dev)
    lut = sb.build_lut(gs, c["key_bits"])
    a, lev = sb.assign_chunks(gt, gs, lut, c["levels"], c["threshold"], c["seed"])
    out = sb.stylize(gt, gs, st, lut, c["levels"], c["threshold"], radius, c["seed"])
    torch.cuda.synchronize()
    return lut, u32(a), lev.cpu().numpy(), out.cpu().numpy()


# ---------------------------------------------------------------------------
# look-up table (Section 3.1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("channels,bits,key_bits,shape", [
    (3, 8, 4, (37, 45)), (2, 8, 6, (64, 64)), (1, 8, 8, (17, 9)), (4, 8, 3, (33, 20)),
    (2, 16, 7, (48, 40)), (1, 16, 10, (30, 31)), (3, 8, 5, (1, 1)), (2, 8, 8, (70, 3)),
    (3, 8, 8, (5, 7))])  # 2^24 bins: every guide value its own bin
def test_lut_all_entries_match_oracle(cuda_device, channels, bits, key_bits, shape):
    H, W = shape
    src = synth.random_guide(1000 + channels * 7 + bits, H, W, channels, bits=bits)
    lut = sb.build_lut(to_dev(src, cuda_device), key_bits)
    got = lut.entries().cpu().numpy().view(np.uint32)
    ref = oracle.build_lut(src, key_bits)
    assert np.array_equal(got, ref)


def test_lut_with_ties_and_constant_regions(cuda_device):
    src = synth.random_guide(5, 50, 41, 2, bits=8, low=100, high=103)  # heavy ties
    src[10:30, 5:25] = 7
    lut = sb.build_lut(to_dev(src, cuda_device), 5)
    assert np.array_equal(lut.entries().cpu().numpy().view(np.uint32),
                          oracle.build_lut(src, 5))


def test_lut_sphere_normals_full_table(cuda_device):
    src = synth.sphere_normals(128)
    lut = sb.build_lut(to_dev(src, cuda_device), 5)
    assert np.array_equal(lut.entries().cpu().numpy().view(np.uint32),
                          oracle.build_lut(src, 5))


@pytest.mark.parametrize("name", ["1080p", "4k"])
def test_lut_full_size_sampled_bins(cuda_device, name):
    w = workload(name)
    ex = w.exemplar
    lut = sb.build_lut(to_dev(ex.guide, cuda_device), ex.lut_bits)
    got = lut.entries().cpu().numpy().view(np.uint32)
    assert got.shape[0] == 1 << (ex.guide.shape[2] * ex.lut_bits)
    rng = np.random.default_rng(7)
    idx = np.concatenate([rng.integers(0, got.shape[0], 160), [0, got.shape[0] - 1]])
    assert np.array_equal(got[idx], oracle.lut_entries(ex.guide, ex.lut_bits, idx))
    # every entry is a valid source position
    assert ((got & 0xFFFF) < ex.guide.shape[1]).all() and ((got >> 16) < ex.guide.shape[0]).all()


# ---------------------------------------------------------------------------
# assignment (Algorithm 2) and fused stylisation, whole small frames
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", REGRESSION_CASES)
def test_small_cases_bit_exact(cuda_device, name):
    c = make_case(name)
    lut, a, lev, out = _full(cuda_device, c)
    ref_out, ref_a, ref_lev = oracle.stylize(c["tgt"], c["src"], c["style"], c["key_bits"],
                                             c["levels"], c["threshold"], c["radius"], c["seed"])
    assert np.array_equal(a, ref_a)
    assert np.array_equal(lev, ref_lev)
    assert np.array_equal(out, ref_out)


@pytest.mark.parametrize("radius", [0, 1, 2, 3, 5, 7, 8, 11, 15])
def test_workload_256_every_radius(cuda_device, radius):
    w = workload("256")
    ex, fr = w.exemplar, w.frames[0]
    c = dict(tgt=fr.guide, src=ex.guide, style=ex.style, key_bits=ex.lut_bits,
             levels=w.levels, threshold=w.threshold, radius=radius, seed=w.seed)
    lut, a, lev, out = _full(cuda_device, c)
    ref_out, ref_a, ref_lev = oracle.stylize(fr.guide, ex.guide, ex.style, ex.lut_bits, w.levels,
                                             w.threshold, radius, w.seed, n_threads=4)
    assert np.array_equal(a, ref_a) and np.array_equal(lev, ref_lev)
    assert np.array_equal(out, ref_out)


@pytest.mark.parametrize("shape,levels,T,seed", [
    ((1, 1), 3, 100, 0), ((1, 97), 4, 50, 1), ((65, 1), 2, 50, 2), ((33, 65), 5, 0, 3),
    ((129, 70), 1, 100, 4), ((70, 129), 12, 200, 5), ((100, 190), 6, (1 << 64) - 1, 6),
    ((64, 32), 7, 400, 0xFFFFFFFF), ((31, 200), 3, 300, 12345),
    # level 8 (the largest level with packed seed keys) with every pixel falling
    # to level 1, level 8 with a mid threshold, level 9 (per-pixel lists)
    ((300, 520), 8, 0, 77), ((97, 203), 8, 2000, 79), ((260, 300), 9, 500, 78),
    # the deepest hierarchies (spacing up to 2^15): on a 50000-pixel-wide target
    # seed distances pass 2^31, so their squared distances need 64 bits
    ((150, 700), 13, 150, 93), ((2, 50000), 15, 300, 91), ((3, 65535), 15, 0, 94)])
def test_ragged_and_extreme_parameters(cuda_device, shape, levels, T, seed):
    H, W = shape
    tgt = synth.smooth_integer_guide(seed % 1000 + 1, H, W, 3, step=5)
    src = synth.smooth_integer_guide(seed % 1000 + 2, 40, 52, 3, step=5)
    style = synth.random_style(seed % 1000 + 3, 40, 52)
    c = dict(tgt=tgt, src=src, style=style, key_bits=5, levels=levels, threshold=T, radius=2,
             seed=seed)
    lut, a, lev, out = _full(cuda_device, c)
    ref_out, ref_a, ref_lev = oracle.stylize(tgt, src, style, 5, levels, T, 2, seed)
    assert np.array_equal(a, ref_a) and np.array_equal(lev, ref_lev)
    assert np.array_equal(out, ref_out)


def test_empty_targets_are_a_no_op(cuda_device):
    src = synth.random_guide(1, 16, 16, 3)
    gs = to_dev(src, cuda_device)
    st = to_dev(synth.random_style(2, 16, 16), cuda_device)
    lut = sb.build_lut(gs, 4)
    for shape in [(0, 0, 3), (0, 9, 3), (9, 0, 3)]:
        gt = torch.zeros(shape, dtype=torch.uint8, device=cuda_device)
        out = sb.stylize(gt, gs, st, lut, 3, 100, 2, 0)
        a, lev = sb.assign_chunks(gt, gs, lut, 3, 100, 0)
        assert out.numel() == 0 and a.numel() == 0
    torch.cuda.synchronize()


def test_identity_uv_reproduces_the_exemplar(cuda_device):
    H, W = 200, 300
    g = synth.identity_uv_guide(H, W)
    style = synth.random_style(9, H, W)
    gd = to_dev(g, cuda_device)
    st = to_dev(style, cuda_device)
    lut = sb.build_lut(gd, 11)
    for radius in (0, 3, 7, 15):
        out = sb.stylize(gd, gd, st, lut, 6, 0, radius, 77)
        assert np.array_equal(out.cpu().numpy(), style)
    a, lev = sb.assign_chunks(gd, gd, lut, 6, 0, 77)
    ys, xs = np.mgrid[0:H, 0:W]
    A = u32(a)
    assert np.array_equal(A & 0xFFFF, xs) and np.array_equal(A >> 16, ys)
    assert (lev.cpu().numpy() == 6).all()


def test_unused_style_rows_and_strided_guides(cuda_device):
    """Row strides larger than the row (a crop of a bigger buffer)."""
    c = make_case("u8x2-33x29-L4-T60-r2")
    big_t = np.zeros((c["tgt"].shape[0], c["tgt"].shape[1] + 7, 2), dtype=np.uint8)
    big_t[:, :c["tgt"].shape[1]] = c["tgt"]
    big_s = np.zeros((c["style"].shape[0], c["style"].shape[1] + 3, 4), dtype=np.uint8)
    big_s[:, :c["style"].shape[1]] = c["style"]
    gt = to_dev(big_t, cuda_device)[:, :c["tgt"].shape[1]]
    gs = to_dev(c["src"], cuda_device)
    st = to_dev(big_s, cuda_device)[:, :c["style"].shape[1]]
    lut = sb.build_lut(gs, c["key_bits"])
    out = sb.stylize(gt, gs, st, lut, c["levels"], c["threshold"], c["radius"], c["seed"])
    ref_out, _, _ = oracle.stylize(c["tgt"], c["src"], c["style"], c["key_bits"], c["levels"],
                                   c["threshold"], c["radius"], c["seed"])
    assert np.array_equal(out.cpu().numpy(), ref_out)


# ---------------------------------------------------------------------------
# voting (Section 3.2) from oracle assignment maps
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("radius", [0, 1, 2, 3, 7, 11, 15])
def test_blend_rgba8_and_f32_match_oracle(cuda_device, radius):
    w = workload("256")
    ex, fr = w.exemplar, w.frames[0]
    a, _ = oracle.assign(fr.guide, ex.guide, ex.lut_bits, w.levels, 60, w.seed, n_threads=4)
    a = a[:150, :201]  # ragged
    ad = torch.from_numpy(a.view(np.int32).copy()).to(cuda_device)
    st = to_dev(ex.style, cuda_device)
    out8 = sb.blend(ad, st, radius)
    outf = sb.blend(ad, st, radius, f32=True)
    torch.cuda.synchronize()
    assert np.array_equal(out8.cpu().numpy(), oracle.blend_rgba8(a, ex.style, radius))
    ref = oracle.blend_f32(a, ex.style, radius)
    assert np.abs(outf.cpu().numpy().astype(np.float64) - ref).max() <= F32_TOL


# ---------------------------------------------------------------------------
# full-size workloads: whole frames against the oracle, in the launch
# configuration the benchmark times (one sb_stylize_batch launch over several
# frames), plus the single-frame and unfused paths and full-frame properties
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,n_frames", [("1080p", 3), ("4k", 2)])
def test_full_size_whole_frames_match_oracle(cuda_device, name, n_frames):
    w = synth.workload_1080p(n_frames) if name == "1080p" else synth.workload_4k_uv(n_frames)
    ex = w.exemplar
    H, W = w.frames[0].guide.shape[:2]
    gs, st = to_dev(ex.guide, cuda_device), to_dev(ex.style, cuda_device)
    lut = sb.build_lut(gs, ex.lut_bits)
    gts = [to_dev(f.guide, cuda_device) for f in w.frames]
    seeds = [w.seed + 7919 * i for i in range(n_frames)]
    batch = sb.stylize_batch([sb.BatchFrame(gts[i], lut, st, w.levels, w.threshold, seeds[i])
                              for i in range(n_frames)], w.blend_radius)
    single = sb.stylize(gts[0], gs, st, lut, w.levels, w.threshold, w.blend_radius, seeds[0])
    maps = [sb.assign_chunks(g, gs, lut, w.levels, w.threshold, s) for g, s in zip(gts, seeds)]
    unfused = sb.blend(maps[0][0], st, w.blend_radius)
    torch.cuda.synchronize()
    ref_lut = oracle.new_lut(ex.guide.shape[2], ex.lut_bits)
    for i, f in enumerate(w.frames):
        ref_out, ref_a, ref_lev = oracle.stylize(f.guide, ex.guide, ex.style, ex.lut_bits,
                                                 w.levels, w.threshold, w.blend_radius, seeds[i],
                                                 lut=ref_lut, n_threads=os.cpu_count() or 1)
        A, lev = u32(maps[i][0]), maps[i][1].cpu().numpy()
        assert np.array_equal(A, ref_a), f"frame {i}: assignment"
        assert np.array_equal(lev, ref_lev), f"frame {i}: levels"
        assert np.array_equal(batch[i].cpu().numpy(), ref_out), f"frame {i}: batched RGBA8"
        if i == 0:
            assert np.array_equal(single.cpu().numpy(), ref_out), "single-frame RGBA8"
            assert np.array_equal(unfused.cpu().numpy(), ref_out), "unfused RGBA8"
            # every accepted candidate above level 1 satisfies the threshold
            Ax, Ay = (A & 0xFFFF).astype(np.int64), (A >> 16).astype(np.int64)
            assert (Ax < ex.guide.shape[1]).all() and (Ay < ex.guide.shape[0]).all()
            d = ((ex.guide[Ay, Ax].astype(np.int64) - f.guide.astype(np.int64)) ** 2).sum(-1)
            assert (d[lev > 1] <= w.threshold).all()
            assert lev.min() >= 1 and lev.max() <= w.levels and (H, W) == A.shape


# ---------------------------------------------------------------------------
# lookup-only comparator (Section 4: texture mapping)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", REGRESSION_CASES)
def test_lookup_only_matches_oracle(cuda_device, case):
    c = make_case(case)
    gt, gs, st = to_dev(c["tgt"], cuda_device), to_dev(c["src"], cuda_device), to_dev(c["style"], cuda_device)
    lut = sb.build_lut(gs, c["key_bits"])
    out = sb.lookup_only(gt, gs, st, lut)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(),
                          oracle.lookup_only(c["tgt"], c["src"], c["style"], c["key_bits"]))


@pytest.mark.parametrize("W,H,channels,offset", [
    (1028, 5, 3, 0),   # four pixels per thread with vector loads; two CTAs per row
    (1030, 7, 3, 0),   # width not a multiple of 4: per-pixel loads
    (515, 3, 2, 1),    # rows start one pixel in: unaligned
    (260, 4, 4, 0), (261, 3, 1, 0),
    (2052, 3, 3, 0),   # rows >= 2048: two quads per thread, the last thread has one
    (2051, 2, 3, 0),   # two quads per thread, per-pixel loads
    (4096, 2, 4, 0)])
def test_lookup_only_vector_and_ragged_rows(cuda_device, W, H, channels, offset):
    """The comparator's vector path (aligned rows, width a multiple of 4) and
    its per-pixel path give the same pixels as the oracle."""
    big = synth.random_guide(W + channels, H, W + offset, channels)
    tgt = np.ascontiguousarray(big)
    src = synth.random_guide(W + 1, 20, 30, channels)
    style = synth.random_style(W + 2, 20, 30)
    gs, st = to_dev(src, cuda_device), to_dev(style, cuda_device)
    lut = sb.build_lut(gs, 5)
    gt = to_dev(tgt, cuda_device)[:, offset:]
    out = sb.lookup_only(gt, gs, st, lut)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), oracle.lookup_only(tgt[:, offset:], src, style, 5))


def test_lookup_only_full_size_sampled(cuda_device):
    w = workload("4k")
    ex, fr = w.exemplar, w.frames[0]
    gs, st = to_dev(ex.guide, cuda_device), to_dev(ex.style, cuda_device)
    lut = sb.build_lut(gs, ex.lut_bits)
    out = sb.lookup_only(to_dev(fr.guide, cuda_device), gs, st, lut).cpu().numpy()
    xs, ys = sample_pixels(3, 3840, 2160, 100)
    for x, y in zip(xs, ys):
        e = oracle.lut_entry(ex.guide, ex.lut_bits, oracle.lut_index(fr.guide, int(x), int(y), ex.lut_bits))
        assert (out[y, x] == ex.style[e >> 16, e & 0xFFFF]).all()


# ---------------------------------------------------------------------------
# keys too wide for a table: the search index (Section 3.1, search trees for
# more guide channels)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("channels,bits,key_bits,radius", [
    (4, 8, 8, 2), (4, 8, 7, 0), (2, 16, 16, 3), (2, 16, 13, 1)])
def test_wide_keys_search_index_matches_oracle(cuda_device, channels, bits, key_bits, radius):
    """Keys of 28-32 bits get a search index instead of a table; every seed's
    u* is then an exact nearest-pixel query.  Assignment, levels and RGBA8
    output (single frame and batched) equal the oracle's, which computes each
    u* from its definition."""
    tgt = synth.smooth_integer_guide(80 + key_bits, 70, 150, channels, step=5)
    src = synth.smooth_integer_guide(90 + key_bits, 45, 61, channels, step=5)
    if bits == 16:
        tgt = tgt.astype(np.uint16) * 257 + 5
        src = src.astype(np.uint16) * 257
    style = synth.random_style(95, 45, 61)
    gt, gs, st = to_dev(tgt, cuda_device), to_dev(src, cuda_device), to_dev(style, cuda_device)
    lut = sb.build_lut(gs, key_bits)
    info = lut.info()
    assert info["entries_ptr"] is None or info["entries_ptr"] == 0
    assert info["n_entries"] == 0
    levels, T, seed = 5, 300 if bits == 8 else 1 << 21, 4242
    a, lev = sb.assign_chunks(gt, gs, lut, levels, T, seed)
    out = sb.stylize(gt, gs, st, lut, levels, T, radius, seed)
    bout = sb.stylize_batch([sb.BatchFrame(gt, lut, st, levels, T, seed)], radius)[0]
    torch.cuda.synchronize()
    ref_out, ref_a, ref_lev = oracle.stylize(tgt, src, style, key_bits, levels, T, radius, seed,
                                             n_threads=4)
    assert np.array_equal(u32(a), ref_a) and np.array_equal(lev.cpu().numpy(), ref_lev)
    assert np.array_equal(out.cpu().numpy(), ref_out)
    assert torch.equal(bout, out)
    with pytest.raises(sb.StyleBlitError) as e:
        sb.lookup_only(gt, gs, st, lut)
    assert e.value.status == -2
    with pytest.raises(ValueError):
        lut.entries()


# ---------------------------------------------------------------------------
# extra guide channels (Section 4 segmentation guide): table keyed on the local guide
# ---------------------------------------------------------------------------

def _segmented(seed, H, W, Hs, Ws):
    GT = synth.smooth_integer_guide(60 + seed, H, W, 4, step=4)
    GS = synth.smooth_integer_guide(70 + seed, Hs, Ws, 4, step=4)
    GT[..., 3] = np.where((np.arange(W)[None, :] // 17 + np.arange(H)[:, None] // 13) % 2, 255, 0)
    GS[..., 3] = np.where(np.arange(Hs)[:, None] < Hs // 2, 0, 255)
    return GT, GS


@pytest.mark.parametrize("kc,kb", [(3, 5), (2, 7), (1, 8)])
def test_keyed_table_matches_oracle(cuda_device, kc, kb):
    _, GS = _segmented(1, 8, 8, 45, 53)
    lut = sb.build_lut(to_dev(GS, cuda_device), kb, key_channels=kc)
    assert lut.info()["key_channels"] == kc and lut.n_entries == 1 << (kc * kb)
    got = lut.entries().cpu().numpy().view(np.uint32)
    assert np.array_equal(got, oracle.build_lut(GS, kb, key_channels=kc))


@pytest.mark.parametrize("radius,T", [(0, 400), (2, 2500), (3, 6000)])
def test_segmentation_guide_stylize_matches_oracle(cuda_device, radius, T):
    GT, GS = _segmented(2, 97, 131, 48, 60)
    style = synth.random_style(5, 48, 60)
    gt, gs, st = to_dev(GT, cuda_device), to_dev(GS, cuda_device), to_dev(style, cuda_device)
    lut = sb.build_lut(gs, 5, key_channels=3)
    a, lev = sb.assign_chunks(gt, gs, lut, 5, T, 9)
    out = sb.stylize(gt, gs, st, lut, 5, T, radius, 9)
    torch.cuda.synchronize()
    ref_out, ref_a, ref_lev = oracle.stylize(GT, GS, style, 5, 5, T, radius, 9, key_channels=3)
    assert np.array_equal(u32(a), ref_a) and np.array_equal(lev.cpu().numpy(), ref_lev)
    assert np.array_equal(out.cpu().numpy(), ref_out)
    A = u32(a)
    L = lev.cpu().numpy()
    seg = GS[A >> 16, A & 0xFFFF, 3]
    assert (seg[L > 1] == GT[..., 3][L > 1]).all()  # no chunk crosses a segment


@pytest.mark.parametrize("tgt_shape,src_shape,levels", [
    ((2, 65535), (3, 32767), 12),   # widest target and source the ABI allows
    ((65535, 2), (32767, 3), 9),    # tallest
])
def test_maximum_target_and_source_sides(cuda_device, tgt_shape, src_shape, levels):
    (Ht, Wt), (Hs, Ws) = tgt_shape, src_shape
    tgt = synth.smooth_integer_guide(91, Ht, Wt, 3, step=7)
    src = synth.smooth_integer_guide(92, Hs, Ws, 3, step=7)
    style = synth.random_style(93, Hs, Ws)
    c = dict(tgt=tgt, src=src, style=style, key_bits=5, levels=levels, threshold=400, radius=2,
             seed=94)
    lut, a, lev, out = _full(cuda_device, c)
    ref_out, ref_a, ref_lev = oracle.stylize(tgt, src, style, 5, levels, 400, 2, 94)
    assert np.array_equal(a, ref_a) and np.array_equal(lev, ref_lev)
    assert np.array_equal(out, ref_out)


@pytest.mark.parametrize("src_shape", [(1, 1), (1, 7), (5, 1), (2, 3)])
def test_degenerate_tiny_sources(cuda_device, src_shape):
    """A source of a pixel or a line: nearly every candidate falls outside it,
    so level 1's clamp decides most pixels; the vote skips out-of-source taps."""
    Hs, Ws = src_shape
    tgt = synth.smooth_integer_guide(71, 45, 70, 3, step=5)
    src = synth.random_guide(72, Hs, Ws, 3)
    style = synth.random_style(73, Hs, Ws)
    c = dict(tgt=tgt, src=src, style=style, key_bits=4, levels=4, threshold=5000, radius=2,
             seed=74)
    lut, a, lev, out = _full(cuda_device, c)
    ref_out, ref_a, ref_lev = oracle.stylize(tgt, src, style, 4, 4, 5000, 2, 74)
    assert np.array_equal(a, ref_a) and np.array_equal(lev, ref_lev)
    assert np.array_equal(out, ref_out)


def _random_case(seed):
    """A seeded random configuration: guide format, sizes, key bits and keyed
    channels, levels, threshold, blend radius, jitter seed."""
    rng = np.random.default_rng(seed)
    channels, bits = [(1, 8), (2, 8), (3, 8), (4, 8), (1, 16), (2, 16)][seed % 6]
    kc = int(rng.integers(1, channels + 1))
    kb_max = min(bits, 24 // kc, 12)
    kb = int(rng.integers(max(1, kb_max - 4), kb_max + 1))
    Ht, Wt = int(rng.integers(1, 140)), int(rng.integers(1, 200))
    Hs, Ws = int(rng.integers(1, 60)), int(rng.integers(1, 60))
    high = (1 << bits) - 1
    tgt = synth.random_guide(10 * seed + 1, Ht, Wt, channels, bits=bits, low=0,
                             high=int(rng.integers(1, high + 1)))
    src = synth.random_guide(10 * seed + 2, Hs, Ws, channels, bits=bits, low=0,
                             high=int(rng.integers(1, high + 1)))
    style = synth.random_style(10 * seed + 3, Hs, Ws)
    T = int(rng.choice([0, int(rng.integers(0, 4 * high * high)), (1 << 64) - 1]))
    return dict(tgt=tgt, src=src, style=style, kb=kb, kc=kc, levels=int(rng.integers(1, 16)),
                T=T, r=int(rng.integers(0, 16)), seed=int(rng.integers(0, 2**32)))


@pytest.mark.parametrize("seed", range(24))
def test_randomized_configurations_match_oracle(cuda_device, seed):
    """Seeded random formats, sizes (ragged, tiny), key bits and keyed channels,
    level counts (1-15), thresholds and radii (0-15): table, assignment, levels and RGBA8
    output equal the oracle's."""
    c = _random_case(seed)
    gt, gs, st = to_dev(c["tgt"], cuda_device), to_dev(c["src"], cuda_device), to_dev(c["style"], cuda_device)
    lut = sb.build_lut(gs, c["kb"], key_channels=c["kc"])
    a, lev = sb.assign_chunks(gt, gs, lut, c["levels"], c["T"], c["seed"])
    out = sb.stylize(gt, gs, st, lut, c["levels"], c["T"], c["r"], c["seed"])
    torch.cuda.synchronize()
    ref_lut = oracle.build_lut(c["src"], c["kb"], key_channels=c["kc"])
    assert np.array_equal(lut.entries().cpu().numpy().view(np.uint32), ref_lut)
    ref_out, ref_a, ref_lev = oracle.stylize(c["tgt"], c["src"], c["style"], c["kb"], c["levels"],
                                             c["T"], c["r"], c["seed"], key_channels=c["kc"])
    assert np.array_equal(u32(a), ref_a) and np.array_equal(lev.cpu().numpy(), ref_lev)
    assert np.array_equal(out.cpu().numpy(), ref_out)


@pytest.mark.parametrize("fmt", range(6))
def test_randomized_mixed_batches_match_oracle(cuda_device, fmt):
    """Four random frames of one guide format, each with its own exemplar, key
    bits, keyed channels, levels, threshold and seed, in one batch under every
    launch schedule: each output equals the oracle's."""
    cases = [_random_case(fmt + 6 * j) for j in range(4)]
    radius = cases[0]["r"]
    luts, frames, refs = [], [], []
    for c in cases:
        lut = sb.build_lut(to_dev(c["src"], cuda_device), c["kb"], key_channels=c["kc"])
        luts.append(lut)
        frames.append((to_dev(c["tgt"], cuda_device), lut, to_dev(c["style"], cuda_device),
                       c["levels"], c["T"], c["seed"]))
        refs.append(oracle.stylize(c["tgt"], c["src"], c["style"], c["kb"], c["levels"], c["T"],
                                   radius, c["seed"], key_channels=c["kc"])[0])
    for persistent in (0, 1):
        for largest_first in (0, 1):
            outs = sb.stylize_batch([sb.BatchFrame(*f) for f in frames], radius,
                                    schedule={"persistent": persistent,
                                              "largest_first": largest_first})
            torch.cuda.synchronize()
            for k, (o, r) in enumerate(zip(outs, refs)):
                assert np.array_equal(o.cpu().numpy(), r), f"schedule {persistent}{largest_first} frame {k}"
    for lut in luts:
        lut.destroy()


@pytest.mark.parametrize("wide", [False, True])
@pytest.mark.parametrize("channels,bits", [(3, 8), (2, 16), (1, 8)])
def test_lookup_only_batch_matches_oracle_and_single_calls(cuda_device, channels, bits, wide):
    """sb_lookup_only_batch: frames of mixed sizes (ragged widths, a row offset
    for the per-pixel path, an empty frame in the middle) over two exemplars
    in one launch; each output equals the oracle's and the single-frame call's."""
    high = (1 << bits) - 1
    exs = []
    for e in range(2):
        src = synth.random_guide(50 + e, 23 + e, 31 + 2 * e, channels, bits=bits, high=high)
        style = synth.random_style(60 + e, 23 + e, 31 + 2 * e)
        gs = to_dev(src, cuda_device)
        exs.append((src, style, gs, to_dev(style, cuda_device), sb.build_lut(gs, 5)))
    shapes = [(37, 1030, 0), (5, 1028, 0), (0, 64, 0), (64, 2051, 1), (1, 1, 0), (33, 260, 0)]
    if wide:  # every frame at least 2048 pixels wide: two quads per thread
        shapes = [(3, 2052, 0), (0, 4096, 0), (2, 4100, 1), (1, 2048, 0)]
    frames, refs, singles = [], [], []
    for i, (h, w, off) in enumerate(shapes):
        src, style, gs, st, lut = exs[i % 2]
        big = synth.random_guide(70 + i, h, w + off, channels, bits=bits, high=high)
        gt = to_dev(big, cuda_device)[:, off:]
        tgt = np.ascontiguousarray(big[:, off:])
        frames.append(sb.BatchFrame(gt, lut, st, 1, 0, 0))
        refs.append(oracle.lookup_only(tgt, src, style, 5))
        singles.append(sb.lookup_only(gt, gs, st, lut))
    outs = sb.lookup_only_batch(frames)
    torch.cuda.synchronize()
    for k, (o, r, s1) in enumerate(zip(outs, refs, singles)):
        assert np.array_equal(o.cpu().numpy(), r), f"frame {k}"
        assert torch.equal(o, s1), f"frame {k}"
    for e in exs:
        e[4].destroy()

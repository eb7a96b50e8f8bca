"""Pins for the oracle's level loop (Algorithm 2, ParallelStyleBlit).

1. An independent, literal Python transcription of Algorithm 2 whose
   u* = argmin_u ||G_T[q] - G_S[u]|| is a brute-force scan of the source (no
   look-up table).  With lossless keys (one table bin per guide value) the
   table lookup must reproduce that argmin exactly, so the two agree pixel by
   pixel.  The transcription carries its own copy of the published fmix32.
2. Invariants that hold for any input: accepted candidates satisfy the
   threshold, identical identity-UV guides reproduce the exemplar, chunks are
   pure translations, acceptance is monotone in the threshold, the extremes
   of threshold and level count.
"""
import numpy as np
import pytest

import oracle
import synth

M32 = 0xFFFFFFFF


def _fmix32(h):
    h ^= h >> 16
    h = (h * 0x85EBCA6B) & M32
    h ^= h >> 13
    h = (h * 0xC2B2AE35) & M32
    h ^= h >> 16
    return h


def _jitter(seed, level, bx, by):
    h = _fmix32(seed ^ ((level * 0x9E3779B9) & M32))
    h = _fmix32(h ^ (bx & M32))
    h = _fmix32(h ^ (by & M32))
    return (h & 0xFFFF) / 65536.0, (h >> 16) / 65536.0


def _seed_point(p, h, level, seed, W, H):
    b = (p[0] // h, p[1] // h)
    j = _jitter(seed, level, *b)
    s = (int(np.floor(h * (b[0] + j[0]))), int(np.floor(h * (b[1] + j[1]))))
    return (min(max(s[0], 0), W - 1), min(max(s[1], 0), H - 1))


def _nearest_seed(p, h, level, seed, W, H):
    d_best, s_best = float("inf"), None
    for x in (-1, 0, 1):
        for y in (-1, 0, 1):
            s = _seed_point((p[0] + h * x, p[1] + h * y), h, level, seed, W, H)
            d = (s[0] - p[0]) ** 2 + (s[1] - p[1]) ** 2
            if d < d_best:
                d_best, s_best = d, s
    return s_best


def _parallel_styleblit(GT, GS, T, L, seed, key_channels=None):
    """Algorithm 2 per pixel, u* by brute-force argmin over all source pixels
    (over the first key_channels channels; the acceptance uses all)."""
    kc = GS.shape[2] if key_channels is None else key_channels
    Ht, Wt = GT.shape[:2]
    Hs, Ws = GS.shape[:2]
    gs = GS.reshape(-1, GS.shape[2]).astype(np.int64)
    A = np.zeros((Ht, Wt, 2), dtype=np.int64)
    lev = np.zeros((Ht, Wt), dtype=np.int64)
    for py in range(Ht):
        for px in range(Wt):
            for level in range(L, 0, -1):
                h = 2 ** level
                q = _nearest_seed((px, py), h, level, seed, Wt, Ht)
                d = ((gs[:, :kc] - GT[q[1], q[0], :kc].astype(np.int64)) ** 2).sum(axis=1)
                u_lin = int(np.argmin(d))  # first minimum = smallest linear index
                u = (u_lin % Ws, u_lin // Ws)
                s = (u[0] + px - q[0], u[1] + py - q[1])
                if level > 1:
                    if not (0 <= s[0] < Ws and 0 <= s[1] < Hs):
                        continue
                    e = ((GS[s[1], s[0]].astype(np.int64) - GT[py, px].astype(np.int64)) ** 2).sum()
                    if e > T:
                        continue
                else:
                    s = (min(max(s[0], 0), Ws - 1), min(max(s[1], 0), Hs - 1))
                A[py, px] = s
                lev[py, px] = level
                break
    return A, lev


def _unpack(a):
    a = a.astype(np.int64)
    return np.stack([a & 0xFFFF, a >> 16], axis=-1)


@pytest.mark.parametrize("case", [
    dict(tgt=(20, 24), src=(12, 16), L=3, T=40, seed=1, smooth=True),
    dict(tgt=(18, 21), src=(16, 16), L=4, T=200, seed=77, smooth=True),
    dict(tgt=(16, 16), src=(10, 9), L=2, T=0, seed=3, smooth=False),
    dict(tgt=(9, 30), src=(20, 6), L=4, T=1000, seed=0xFFFFFFFF, smooth=False),
    dict(tgt=(15, 13), src=(15, 13), L=1, T=50, seed=5, smooth=True),
])
def test_level_loop_matches_literal_algorithm2(case):
    Ht, Wt = case["tgt"]
    Hs, Ws = case["src"]
    if case["smooth"]:
        GT = synth.smooth_integer_guide(10 + case["seed"] % 97, Ht, Wt, 2, step=4)
        GS = synth.smooth_integer_guide(20 + case["seed"] % 89, Hs, Ws, 2, step=4)
    else:
        GT = synth.random_guide(30, Ht, Wt, 2, low=0, high=40)
        GS = synth.random_guide(31, Hs, Ws, 2, low=0, high=40)
    A_ref, lev_ref = _parallel_styleblit(GT, GS, case["T"], case["L"], case["seed"])
    a, lev = oracle.assign(GT, GS, 8, case["L"], case["T"], case["seed"])
    assert np.array_equal(_unpack(a), A_ref)
    assert np.array_equal(lev.astype(np.int64), lev_ref)
    if case["L"] > 1:
        assert len(np.unique(lev_ref)) >= 1


def _guide_dist(GS, GT, a):
    A = _unpack(a)
    s = GS[A[..., 1], A[..., 0]].astype(np.int64)
    return ((s - GT.astype(np.int64)) ** 2).sum(axis=-1)


@pytest.mark.parametrize("channels,bits,T,seed", [(4, 8, 300, 4), (2, 16, 1 << 20, 9)])
def test_wide_keys_without_a_table_match_literal_algorithm2(channels, bits, T, seed):
    """Keys too wide for a table (4 x 8 and 2 x 16 bits, lossless): the oracle
    computes u* from its definition at every seed, which must equal the
    transcription's brute-force argmin."""
    GT = synth.smooth_integer_guide(40 + seed, 17, 22, channels, step=5)
    GS = synth.smooth_integer_guide(50 + seed, 11, 13, channels, step=5)
    if bits == 16:  # spread over 16 bits (and off the multiples of 257 for the target)
        GT = GT.astype(np.uint16) * 257 + 3
        GS = GS.astype(np.uint16) * 257
    assert oracle.new_lut(channels, bits) is None
    A_ref, lev_ref = _parallel_styleblit(GT, GS, T, 4, seed)
    a, lev = oracle.assign(GT, GS, bits, 4, T, seed)
    assert np.array_equal(_unpack(a), A_ref)
    assert np.array_equal(lev, lev_ref)


def test_accepted_candidates_satisfy_threshold_normals():
    w = synth.workload_256()
    ex, fr = w.exemplar, w.frames[0]
    for T in (0, 50, 300, 3000):
        a, lev = oracle.assign(fr.guide, ex.guide, ex.lut_bits, w.levels, T, w.seed, n_threads=4)
        d = _guide_dist(ex.guide, fr.guide, a)
        assert (d[lev > 1] <= T).all()
        A = _unpack(a)
        assert (A[..., 0] < ex.guide.shape[1]).all() and (A[..., 1] < ex.guide.shape[0]).all()


def test_acceptance_is_monotone_in_threshold():
    w = synth.workload_256()
    ex, fr = w.exemplar, w.frames[0]
    prev = None
    for T in (0, 30, 100, 300, 1000, 10000):
        _, lev = oracle.assign(fr.guide, ex.guide, ex.lut_bits, w.levels, T, w.seed, n_threads=4)
        if prev is not None:
            assert (lev >= prev).all()
        prev = lev
    assert prev.mean() > 3.0


def test_threshold_extremes_and_single_level():
    w = synth.workload_256()
    ex, fr = w.exemplar, w.frames[0]
    _, lev = oracle.assign(fr.guide, ex.guide, ex.lut_bits, 1, 0, w.seed)
    assert (lev == 1).all()
    a, lev = oracle.assign(fr.guide, ex.guide, ex.lut_bits, 4, (1 << 64) - 1, w.seed, n_threads=4)
    # with an unbounded threshold only an out-of-source candidate can fall through
    xs, ys = np.nonzero(lev.T != 4)
    for x, y in zip(xs[:200], ys[:200]):
        qx, qy = oracle.nearest_seed(int(x), int(y), 4, w.seed, 256, 256)
        u = oracle.lut_entry(ex.guide, ex.lut_bits, oracle.lut_index(fr.guide, qx, qy, ex.lut_bits))
        sx, sy = (u & 0xFFFF) + x - qx, (u >> 16) + y - qy
        assert not (0 <= sx < 256 and 0 <= sy < 256)
    assert (lev == 4).mean() > 0.9


@pytest.mark.parametrize("L", [1, 3, 5])
def test_identical_identity_uv_guides_reproduce_the_style(L):
    """G_T = G_S = (x << 5, y << 5) with 11-bit keys (one guide value per bin):
    every seed maps onto itself, every candidate is p itself, so A(p) = p at
    the top level even with threshold 0, and every vote returns C_S[p]."""
    H, W = 40, 56
    G = synth.identity_uv_guide(H, W)
    style = synth.random_style(8, H, W)
    a, lev = oracle.assign(G, G, 11, L, 0, 1234)
    A = _unpack(a)
    ys, xs = np.mgrid[0:H, 0:W]
    assert np.array_equal(A[..., 0], xs) and np.array_equal(A[..., 1], ys)
    assert (lev == L).all()
    for r in (0, 1, 3):
        assert np.array_equal(oracle.blend_rgba8(a, style, r), style)


def test_chunks_are_pure_translations():
    """Pixels that share a level and a nearest seed copy one translated chunk:
    A(p) - p is the same for all of them (level 1 excepted, which clamps)."""
    w = synth.workload_256()
    ex, fr = w.exemplar, w.frames[0]
    a, lev = oracle.assign(fr.guide, ex.guide, ex.lut_bits, w.levels, w.threshold, w.seed,
                           n_threads=4)
    A = _unpack(a)
    groups = {}
    for y in range(0, 256, 2):
        for x in range(0, 256, 2):
            l = int(lev[y, x])
            if l == 1:
                continue
            q = oracle.nearest_seed(x, y, l, w.seed, 256, 256)
            d = (int(A[y, x, 0]) - x, int(A[y, x, 1]) - y)
            groups.setdefault((l, q), set()).add(d)
    assert len(groups) > 20
    assert all(len(v) == 1 for v in groups.values())


def test_points_api_matches_full_frame():
    w = synth.workload_256()
    ex, fr = w.exemplar, w.frames[0]
    out, a, lev = oracle.stylize(fr.guide, ex.guide, ex.style, ex.lut_bits, w.levels,
                                 w.threshold, 2, w.seed, n_threads=4)
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.integers(0, 256, 200), [0, 255, 0, 255]])
    ys = np.concatenate([rng.integers(0, 256, 200), [0, 0, 255, 255]])
    pa, pl = oracle.assign_points(fr.guide, ex.guide, ex.lut_bits, w.levels, w.threshold,
                                  w.seed, xs, ys)
    assert np.array_equal(pa, a[ys, xs]) and np.array_equal(pl, lev[ys, xs])
    po = oracle.stylize_points(fr.guide, ex.guide, ex.style, ex.lut_bits, w.levels,
                               w.threshold, 2, w.seed, xs, ys)
    assert np.array_equal(po, out[ys, xs])


@pytest.mark.parametrize("T,seed", [(100, 3), (900, 11)])
def test_segmentation_channel_keys_and_acceptance(T, seed):
    """Section 4 adds a segmentation guide: the table is keyed on the local
    guide only (first two channels here), the acceptance distance includes the
    segment channel (0 or 255).  Literal transcription agrees, and with
    T < 255^2 no accepted chunk crosses a segment boundary."""
    Ht, Wt, Hs, Ws = 22, 26, 16, 18
    GT = synth.smooth_integer_guide(40 + seed, Ht, Wt, 3, step=4)
    GS = synth.smooth_integer_guide(50 + seed, Hs, Ws, 3, step=4)
    GT[..., 2] = np.where(np.arange(Wt)[None, :] < Wt // 2, 0, 255)
    GS[..., 2] = np.where(np.arange(Hs)[:, None] < Hs // 3, 255, 0)
    A_ref, lev_ref = _parallel_styleblit(GT, GS, T, 4, seed, key_channels=2)
    a, lev = oracle.assign(GT, GS, 8, 4, T, seed, key_channels=2)
    assert np.array_equal(_unpack(a), A_ref) and np.array_equal(lev.astype(np.int64), lev_ref)
    A = _unpack(a)
    seg_src = GS[A[..., 1], A[..., 0], 2]
    assert (seg_src[lev > 1] == GT[..., 2][lev > 1]).all()
    # keying on every channel gives a different (larger) table and, here, a different result
    a_all, _ = oracle.assign(GT, GS, 8, 4, T, seed)
    assert not np.array_equal(a_all, a)

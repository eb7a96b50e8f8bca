"""Pins for the oracle's voting step (end of §3.2: coordinates are transferred,
then a target pixel takes the average colour of the co-located pixels of all
source patches covering it).

The oracle sums C_S[A(p + o) - o] over window offsets o.  Writing
A(n) = n + delta(n) turns each term into C_S[p + delta(p + o)], so the same
sum is "count of each distinct translation in the window times the colour at
p + delta" -- a different formula, computed here with numpy, that must agree
exactly in integers.  Hand-worked rounding cases and closed-form special
cases (constant style, radius 0, chunk interiors) complete the pins.
"""
import numpy as np
import pytest

import oracle
import synth


def _pack(x, y):
    return (np.asarray(x, np.uint32) | (np.asarray(y, np.uint32) << 16)).astype(np.uint32)


def _vote_by_translations(A, style, r):
    """Sum over distinct translations delta in the window of count * C_S[p + delta]."""
    H, W = A.shape
    Hs, Ws = style.shape[:2]
    ax = (A & 0xFFFF).astype(np.int64)
    ay = (A >> 16).astype(np.int64)
    ys, xs = np.mgrid[0:H, 0:W]
    dx, dy = ax - xs, ay - ys
    sums = np.zeros((H, W, 4), dtype=np.int64)
    cnt = np.zeros((H, W), dtype=np.int64)
    for y in range(H):
        for x in range(W):
            y0, y1 = max(0, y - r), min(H, y + r + 1)
            x0, x1 = max(0, x - r), min(W, x + r + 1)
            ds = list(zip(dx[y0:y1, x0:x1].ravel(), dy[y0:y1, x0:x1].ravel()))
            for (ddx, ddy) in set(ds):
                k = ds.count((ddx, ddy))
                vx, vy = x + ddx, y + ddy
                if 0 <= vx < Ws and 0 <= vy < Hs:
                    sums[y, x] += k * style[vy, vx].astype(np.int64)
                    cnt[y, x] += k
    return sums, cnt


@pytest.mark.parametrize("r", [0, 1, 2, 3])
def test_vote_equals_translation_histogram_form(r):
    rng = np.random.default_rng(r)
    H, W, Hs, Ws = 14, 17, 12, 15
    style = synth.random_style(40 + r, Hs, Ws)
    # piecewise-constant translations (chunks) plus random noise pixels
    ys, xs = np.mgrid[0:H, 0:W]
    tx = rng.integers(-5, 5, size=(3, 3))[np.minimum(ys // 5, 2), np.minimum(xs // 6, 2)]
    ty = rng.integers(-5, 5, size=(3, 3))[np.minimum(ys // 5, 2), np.minimum(xs // 6, 2)]
    ax = np.clip(xs + tx, 0, Ws - 1)
    ay = np.clip(ys + ty, 0, Hs - 1)
    noise = rng.random((H, W)) < 0.15
    ax[noise] = rng.integers(0, Ws, noise.sum())
    ay[noise] = rng.integers(0, Hs, noise.sum())
    A = _pack(ax, ay)
    sums, cnt = _vote_by_translations(A, style, r)
    out = oracle.blend_rgba8(A, style, r)
    assert (cnt >= 1).all()
    expect = (sums + cnt[..., None] // 2) // cnt[..., None]
    assert np.array_equal(out.astype(np.int64), expect)
    f = oracle.blend_f32(A, style, r)
    assert np.allclose(f * 255.0 * cnt[..., None], sums, rtol=0, atol=1e-9)


def test_radius_zero_copies_and_constant_style_is_constant():
    rng = np.random.default_rng(1)
    H, W = 9, 11
    style = synth.random_style(3, 7, 8)
    A = _pack(rng.integers(0, 8, (H, W)), rng.integers(0, 7, (H, W)))
    out = oracle.blend_rgba8(A, style, 0)
    assert np.array_equal(out, style[A >> 16, A & 0xFFFF])
    const = np.empty_like(style)
    const[...] = [17, 200, 3, 255]
    for r in (1, 2, 4):
        assert (oracle.blend_rgba8(A, const, r) == [17, 200, 3, 255]).all()


def test_chunk_interior_vote_is_a_plain_copy():
    """Blending acts only at chunk boundaries: a pixel whose whole window lies
    in one chunk (one translation) receives the copied colour unchanged."""
    H, W, Hs, Ws = 20, 20, 30, 30
    style = synth.random_style(5, Hs, Ws)
    ys, xs = np.mgrid[0:H, 0:W]
    left = xs < 10
    A = _pack(np.where(left, xs + 3, xs + 7), np.where(left, ys + 2, ys + 9))
    out = oracle.blend_rgba8(A, style, 2)
    copy = style[A >> 16, A & 0xFFFF]
    interior = (xs >= 2) & (xs <= 7) | (xs >= 12) & (xs <= 17)
    assert np.array_equal(out[interior], copy[interior])
    assert not np.array_equal(out[~interior], copy[~interior])


def test_round_half_up_worked_example():
    """1 x 2 target, radius 1, style 1 x 4.  A(0) = 1, A(1) = 3.
    Pixel 0: o=0 -> C_S[1]; o=+1 -> A(1) - 1 = 2 -> C_S[2]; o=-1 outside.
    Pixel 1: o=-1 -> A(0) + 1 = 2 -> C_S[2]; o=0 -> C_S[3]; o=+1 outside.
    Red channel C_S = [0, 10, 11, 200]: pixel 0 = (10 + 11)/2 = 10.5 -> 11,
    pixel 1 = (11 + 200)/2 = 105.5 -> 106."""
    style = np.zeros((1, 4, 4), dtype=np.uint8)
    style[0, :, 0] = [0, 10, 11, 200]
    style[0, :, 1] = [0, 1, 2, 3]      # (1 + 2)/2 = 1.5 -> 2 ; (2 + 3)/2 = 2.5 -> 3
    style[0, :, 3] = 255
    A = _pack([[1, 3]], [[0, 0]])
    out = oracle.blend_rgba8(A, style, 1)
    assert out[0, 0].tolist() == [11, 2, 0, 255]
    assert out[0, 1].tolist() == [106, 3, 0, 255]
    f = oracle.blend_f32(A, style, 1)
    assert f[0, 0, 0] == pytest.approx(21 / 510) and f[0, 1, 0] == pytest.approx(211 / 510)


def test_sources_outside_the_exemplar_are_skipped():
    """A(0) = 0 at the left edge: o = +1 neighbour points to x = -1 + ... ."""
    style = np.zeros((1, 3, 4), dtype=np.uint8)
    style[0, :, 0] = [30, 60, 90]
    # A(0)=0, A(1)=0 -> for p=0, o=+1: A(1) - 1 = -1 (outside): skipped
    A = _pack([[0, 0]], [[0, 0]])
    out = oracle.blend_rgba8(A, style, 1)
    # p=0: only o=0 -> 30. p=1: o=-1 -> A(0)+1 = 1 -> 60; o=0 -> 0 -> 30: 45
    assert out[0, 0, 0] == 30 and out[0, 1, 0] == 45

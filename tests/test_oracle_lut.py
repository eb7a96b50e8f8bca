"""Pins for the oracle's guide look-up table (§3.1: a guide value names a
source position through a simple look-up table).

Pinned by: closed forms of the bin key and representative, the closed form of
the table of an identity-UV source, exact hits, and an independent nearest-
neighbour library routine (scipy's k-d tree) for the minimal distance.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("bits,key_bits", [(8, 8), (8, 6), (8, 4), (16, 10), (16, 11), (16, 16)])
def test_bin_representative_is_floor_of_bin_centre(bits, key_bits):
    width = 1 << (bits - key_bits)
    for key in [0, 1, 2, (1 << key_bits) - 1]:
        rep = oracle.bin_representative(key, 1, bits, key_bits)[0]
        lo, hi = key * width, key * width + width - 1
        assert rep == (lo + hi) // 2
        assert lo <= rep <= hi


def test_lut_index_concatenates_channel_keys_low_first():
    g = np.zeros((1, 1, 3), dtype=np.uint8)
    g[0, 0] = [0b10110111, 0b01000001, 0b11111100]
    # 6-bit keys: drop 2 low bits of each channel
    k0, k1, k2 = 0b101101, 0b010000, 0b111111
    assert oracle.lut_index(g, 0, 0, 6) == k0 | (k1 << 6) | (k2 << 12)
    g16 = np.array([[[0xABCD, 0x1234]]], dtype=np.uint16)
    assert oracle.lut_index(g16, 0, 0, 10) == (0xABCD >> 6) | ((0x1234 >> 6) << 10)


def _nearest_multiple_index(rep, n, step=32):
    """argmin_x |x*step - rep| over 0 <= x < n, ties to the smaller x."""
    q = Fraction(rep, step)
    lo = int(q)  # floor for rep >= 0
    cands = [c for c in (lo, lo + 1) if 0 <= c < n] or [n - 1]
    best = min(cands, key=lambda c: (abs(c * step - rep), c))
    return min(max(best, 0), n - 1)


@pytest.mark.parametrize("key_bits", [10, 11])
def test_identity_uv_source_closed_form(key_bits):
    """Source guide (x << 5, y << 5): the distance separates per channel, so
    the entry is the nearest multiple of 32 per axis (ties to the smaller)."""
    W, H = 64, 48
    src = synth.identity_uv_guide(H, W)
    rng = np.random.default_rng(3)
    idxs = rng.integers(0, 1 << (2 * key_bits), size=300)
    got = oracle.lut_entries(src, key_bits, idxs)
    for idx, e in zip(idxs, got):
        rx, ry = oracle.bin_representative(int(idx), 2, 16, key_bits)
        assert int(e) & 0xFFFF == _nearest_multiple_index(rx, W)
        assert int(e) >> 16 == _nearest_multiple_index(ry, H)
    if key_bits == 10:
        # 10 bits/channel: rep = 64 key + 31, nearest x*32 is x = 2 key + 1
        for key in range(0, 31):
            e = oracle.lut_entry(src, 10, key | (key << 10))
            assert (e & 0xFFFF, e >> 16) == (2 * key + 1, min(2 * key + 1, H - 1))


def test_exact_hits_take_the_first_pixel_in_raster_order():
    # lossless keys (key_bits == bits): representative == guide value
    src = synth.random_guide(11, 9, 13, 2, bits=8, low=0, high=7)  # many repeats
    for y in range(9):
        for x in range(13):
            idx = oracle.lut_index(src, x, y, 8)
            e = oracle.lut_entry(src, 8, idx)
            ex, ey = e & 0xFFFF, e >> 16
            assert (src[ey, ex] == src[y, x]).all()
            # no earlier pixel in raster order holds the same value
            first = np.flatnonzero((src.reshape(-1, 2) == src[y, x]).all(axis=1))[0]
            assert ey * 13 + ex == first


@pytest.mark.parametrize("channels,bits,key_bits,shape", [
    (3, 8, 4, (24, 20)), (2, 8, 5, (17, 31)), (2, 16, 6, (16, 16)), (1, 8, 8, (7, 5)),
    (4, 8, 3, (12, 12)),
    # keys wider than a table (the paper's search-tree case): 28 and 32 bits
    (4, 8, 7, (9, 11)), (4, 8, 8, (12, 14)), (2, 16, 16, (10, 12))])
def test_min_distance_matches_kdtree(channels, bits, key_bits, shape):
    spatial = pytest.importorskip("scipy.spatial")
    H, W = shape
    src = synth.random_guide(100 + channels, H, W, channels, bits=bits)
    pts = src.reshape(-1, channels).astype(np.float64)
    tree = spatial.cKDTree(pts)
    nb = 1 << (channels * key_bits)
    idxs = np.arange(nb) if nb <= 4096 else np.random.default_rng(0).integers(0, nb, 2000)
    got = oracle.lut_entries(src, key_bits, idxs)
    reps = np.array([oracle.bin_representative(int(i), channels, bits, key_bits)
                     for i in idxs], dtype=np.float64)
    dist, _ = tree.query(reps, k=1)
    ex = got & 0xFFFF
    ey = got >> 16
    chosen = src[ey, ex].astype(np.int64)
    d_got = ((chosen - reps.astype(np.int64)) ** 2).sum(axis=1)
    assert np.array_equal(d_got, np.rint(dist ** 2).astype(np.int64))
    # tie rule: the chosen pixel is the first in raster order at that distance
    allp = src.reshape(-1, channels).astype(np.int64)
    for r, e_lin, d in zip(reps.astype(np.int64)[:300], (ey * W + ex)[:300], d_got[:300]):
        dd = ((allp - r) ** 2).sum(axis=1)
        assert np.flatnonzero(dd == d)[0] == e_lin


def test_full_build_equals_entries_and_lazy_fill():
    src = synth.random_guide(5, 10, 14, 3, bits=8)
    full = oracle.build_lut(src, 3, n_threads=2)
    assert full.shape == (1 << 9,)
    assert np.array_equal(full, oracle.lut_entries(src, 3, np.arange(1 << 9)))
    tgt = synth.random_guide(6, 12, 12, 3, bits=8)
    lazy = oracle.new_lut(3, 3)
    a1, l1 = oracle.assign(tgt, src, 3, 3, 200, 9, lut=lazy)
    a2, l2 = oracle.assign(tgt, src, 3, 3, 200, 9, lut=full.copy())
    assert np.array_equal(a1, a2) and np.array_equal(l1, l2)
    filled = lazy != oracle.UNSET
    assert filled.any() and np.array_equal(lazy[filled], full[filled])


def test_lookup_only_closed_forms():
    """The texture-mapping comparator: identical identity-UV guides with one
    guide value per bin return the exemplar itself; a constant target guide
    returns one constant colour, the style at that value's table entry."""
    H, W = 24, 40
    G = synth.identity_uv_guide(H, W)
    style = synth.random_style(2, H, W)
    assert np.array_equal(oracle.lookup_only(G, G, style, 11), style)
    src = synth.random_guide(3, 20, 30, 3)
    st = synth.random_style(4, 20, 30)
    tgt = np.empty((7, 9, 3), np.uint8)
    tgt[...] = [10, 200, 77]
    out = oracle.lookup_only(tgt, src, st, 5)
    e = oracle.lut_entry(src, 5, oracle.lut_index(tgt, 0, 0, 5))
    assert (out == st[e >> 16, e & 0xFFFF]).all()


def test_key_channels_subset_matches_kdtree_on_those_channels():
    """A table keyed on the first key_channels channels maps a bin to the pixel
    nearest in those channels only (the rest are for acceptance)."""
    spatial = pytest.importorskip("scipy.spatial")
    src = synth.random_guide(77, 20, 25, 4, bits=8)
    kc, kb = 2, 6
    idxs = np.arange(1 << (kc * kb))
    got = oracle.lut_entries(src, kb, idxs, key_channels=kc)
    reps = np.array([oracle.bin_representative(int(i), kc, 8, kb) for i in idxs], np.int64)
    dist, _ = spatial.cKDTree(src[..., :kc].reshape(-1, kc).astype(np.float64)).query(reps)
    chosen = src[got >> 16, got & 0xFFFF, :kc].astype(np.int64)
    assert np.array_equal(((chosen - reps) ** 2).sum(1), np.rint(dist ** 2).astype(np.int64))
    assert oracle.lut_index(src, 3, 4, kb, key_channels=kc) < (1 << (kc * kb))
    full = oracle.build_lut(src, kb, key_channels=kc)
    assert np.array_equal(full, got)

"""StyleBlit CPU oracle -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.

A ctypes front end to `styleblit_oracle.c`, the plain scalar C restatement of
the StyleBlit method (Sýkora et al., EGSR 2018): the guide look-up table of
§3.1, Algorithm 2 (ParallelStyleBlit) and the voting step of §3.2.  Only the
test suite, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg may
import this package.  It shares no code with the CUDA library.

Every function here takes numpy arrays in interleaved HWC layout and returns
numpy arrays; look-up tables are uint32 arrays of 2^(channels * key_bits)
entries packed x | y << 16, where the value 0xFFFFFFFF marks an entry not yet
computed (the oracle fills those on first use).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "styleblit_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

UNSET = 0xFFFFFFFF
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-Wall", "-Wextra", _SRC, "-o", tmp]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Guide(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("channels", ctypes.c_int32),
                ("bits", ctypes.c_int32), ("row_stride", ctypes.c_int64)]


class _Rgba8(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("row_stride", ctypes.c_int64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            u32, i32, i64, u64 = ctypes.c_uint32, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
            vp = ctypes.c_void_p
            sig = {
                "orc_fmix32": (u32, [u32]),
                "orc_cell_hash": (u32, [u32, i32, i32, i32]),
                "orc_lut_index": (u32, [P(_Guide), i32, i32, i32]),
                "orc_bin_representative": (None, [u32, i32, i32, i32, P(u32)]),
                "orc_lut_entry": (u32, [P(_Guide), i32, u32]),
                "orc_lut_entry_k": (u32, [P(_Guide), i32, i32, u32]),
                "orc_lut_index_k": (u32, [P(_Guide), i32, i32, i32, i32]),
                "orc_build_lut": (ctypes.c_int, [P(_Guide), i32, i32, vp, i32]),
                "orc_seed_point": (None, [i64, i64, i32, u32, i32, i32, P(i64), P(i64)]),
                "orc_nearest_seed": (None, [i32, i32, i32, u32, i32, i32, P(i32), P(i32)]),
                "orc_assign": (ctypes.c_int, [P(_Guide), P(_Guide), i32, i32, vp, i32, u64,
                                              u32, vp, vp, i32]),
                "orc_assign_points": (ctypes.c_int, [P(_Guide), P(_Guide), i32, i32, vp, i32,
                                                     u64, u32, vp, vp, i64, vp, vp]),
                "orc_blend_rgba8": (ctypes.c_int, [vp, i32, i32, P(_Rgba8), i32, vp, i32]),
                "orc_blend_f32": (ctypes.c_int, [vp, i32, i32, P(_Rgba8), i32, vp, i32]),
                "orc_stylize_points": (ctypes.c_int, [P(_Guide), P(_Guide), P(_Rgba8), i32, i32,
                                                      vp, i32, u64, i32, u32, vp, vp, i64,
                                                      vp]),
                "orc_lookup_only": (ctypes.c_int, [P(_Guide), P(_Guide), P(_Rgba8), i32, i32, vp,
                                                   vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _guide(a: np.ndarray) -> tuple[_Guide, np.ndarray]:
    if a.ndim == 2:
        a = a[:, :, None]
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint8:
        bits = 8
    elif a.dtype == np.uint16:
        bits = 16
    else:
        raise TypeError(f"guide dtype must be uint8 or uint16, got {a.dtype}")
    h, w, c = a.shape
    return _Guide(a.ctypes.data, w, h, c, bits, a.strides[0]), a


def _style(a: np.ndarray) -> tuple[_Rgba8, np.ndarray]:
    a = np.ascontiguousarray(a, dtype=np.uint8)
    if a.ndim != 3 or a.shape[2] != 4:
        raise ValueError("style must be uint8 [H, W, 4]")
    h, w, _ = a.shape
    return _Rgba8(a.ctypes.data, w, h, a.strides[0]), a


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# --------------------------------------------------------------------------
# hash and seeds (Algorithm 2: SeedPoint, NearestSeed)
# --------------------------------------------------------------------------

def fmix32(h: int) -> int:
    return int(_load().orc_fmix32(h & 0xFFFFFFFF))


def cell_hash(seed: int, level: int, bx: int, by: int) -> int:
    return int(_load().orc_cell_hash(seed & 0xFFFFFFFF, level, bx, by))


def seed_point(px: int, py: int, level: int, seed: int, tgt_w: int, tgt_h: int):
    sx, sy = ctypes.c_int64(), ctypes.c_int64()
    _load().orc_seed_point(px, py, level, seed & 0xFFFFFFFF, tgt_w, tgt_h,
                           ctypes.byref(sx), ctypes.byref(sy))
    return sx.value, sy.value


def nearest_seed(px: int, py: int, level: int, seed: int, tgt_w: int, tgt_h: int):
    qx, qy = ctypes.c_int32(), ctypes.c_int32()
    _load().orc_nearest_seed(px, py, level, seed & 0xFFFFFFFF, tgt_w, tgt_h,
                             ctypes.byref(qx), ctypes.byref(qy))
    return qx.value, qy.value


# --------------------------------------------------------------------------
# look-up table (§3.1)
# --------------------------------------------------------------------------

def lut_size(channels: int, key_bits: int) -> int:
    return 1 << (channels * key_bits)


TABLE_MAX_KEY_BITS = 24


def new_lut(channels: int, key_bits: int) -> np.ndarray | None:
    """An empty table: every entry is computed on first use.  Keys wider than
    24 bits get no table (None): every use computes the entry from its
    definition."""
    if channels * key_bits > TABLE_MAX_KEY_BITS:
        return None
    return np.full(lut_size(channels, key_bits), UNSET, dtype=np.uint32)


def _lut_ptr(lut):
    return None if lut is None else _ptr(lut)


def lut_index(guide: np.ndarray, x: int, y: int, key_bits: int, key_channels=None) -> int:
    g, keep = _guide(guide)
    kc = g.channels if key_channels is None else key_channels
    return int(_load().orc_lut_index_k(ctypes.byref(g), x, y, key_bits, kc))


def bin_representative(idx: int, channels: int, bits: int, key_bits: int) -> list[int]:
    rep = (ctypes.c_uint32 * 4)()
    _load().orc_bin_representative(idx, channels, bits, key_bits, rep)
    return [int(rep[c]) for c in range(channels)]


def lut_entry(src_guide: np.ndarray, key_bits: int, idx: int, key_channels=None) -> int:
    g, keep = _guide(src_guide)
    kc = g.channels if key_channels is None else key_channels
    return int(_load().orc_lut_entry_k(ctypes.byref(g), key_bits, kc, idx))


def lut_entries(src_guide: np.ndarray, key_bits: int, idxs, key_channels=None) -> np.ndarray:
    g, keep = _guide(src_guide)
    kc = g.channels if key_channels is None else key_channels
    lib = _load()
    return np.array([lib.orc_lut_entry_k(ctypes.byref(g), key_bits, kc, int(i)) for i in idxs],
                    dtype=np.uint32)


def build_lut(src_guide: np.ndarray, key_bits: int, n_threads: int = 0,
              key_channels=None) -> np.ndarray:
    g, keep = _guide(src_guide)
    kc = g.channels if key_channels is None else key_channels
    if kc * key_bits > TABLE_MAX_KEY_BITS:
        raise ValueError("keys wider than 24 bits have no table; use lut_entries")
    lut = np.empty(lut_size(kc, key_bits), dtype=np.uint32)
    _load().orc_build_lut(ctypes.byref(g), key_bits, kc, _ptr(lut), n_threads or os.cpu_count())
    return lut


# --------------------------------------------------------------------------
# Algorithm 2 level loop and the vote of §3.2
# --------------------------------------------------------------------------

def assign(tgt_guide, src_guide, key_bits, levels, threshold, seed, lut=None, n_threads=1,
           key_channels=None):
    """Chunk assignment of every target pixel: (A packed x|y<<16, level)."""
    t, kt = _guide(tgt_guide)
    s, ks = _guide(src_guide)
    kc = s.channels if key_channels is None else key_channels
    if lut is None:
        lut = new_lut(kc, key_bits)
    a = np.empty((t.height, t.width), dtype=np.uint32)
    lev = np.empty((t.height, t.width), dtype=np.uint8)
    _load().orc_assign(ctypes.byref(t), ctypes.byref(s), key_bits, kc, _lut_ptr(lut), levels,
                       int(threshold), seed & 0xFFFFFFFF, _ptr(a), _ptr(lev), n_threads)
    return a, lev


def assign_points(tgt_guide, src_guide, key_bits, levels, threshold, seed, xs, ys, lut=None,
                  key_channels=None):
    t, kt = _guide(tgt_guide)
    s, ks = _guide(src_guide)
    kc = s.channels if key_channels is None else key_channels
    if lut is None:
        lut = new_lut(kc, key_bits)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    a = np.empty(len(xs), dtype=np.uint32)
    lev = np.empty(len(xs), dtype=np.uint8)
    _load().orc_assign_points(ctypes.byref(t), ctypes.byref(s), key_bits, kc, _lut_ptr(lut), levels,
                              int(threshold), seed & 0xFFFFFFFF, _ptr(xs), _ptr(ys), len(xs),
                              _ptr(a), _ptr(lev))
    return a, lev


def blend_rgba8(assign_map, style, radius, n_threads=1):
    a = np.ascontiguousarray(assign_map, dtype=np.uint32)
    st, ks = _style(style)
    h, w = a.shape
    out = np.empty((h, w, 4), dtype=np.uint8)
    _load().orc_blend_rgba8(_ptr(a), w, h, ctypes.byref(st), radius, _ptr(out), n_threads)
    return out


def blend_f32(assign_map, style, radius, n_threads=1):
    """Float vote: sum / (255 n), computed in double."""
    a = np.ascontiguousarray(assign_map, dtype=np.uint32)
    st, ks = _style(style)
    h, w = a.shape
    out = np.empty((h, w, 4), dtype=np.float64)
    _load().orc_blend_f32(_ptr(a), w, h, ctypes.byref(st), radius, _ptr(out), n_threads)
    return out


def stylize(tgt_guide, src_guide, style, key_bits, levels, threshold, radius, seed,
            lut=None, n_threads=1, key_channels=None):
    """Full frame: assignment, then the RGBA8 vote."""
    a, lev = assign(tgt_guide, src_guide, key_bits, levels, threshold, seed, lut, n_threads,
                    key_channels)
    return blend_rgba8(a, style, radius, n_threads), a, lev


def stylize_points(tgt_guide, src_guide, style, key_bits, levels, threshold, radius, seed,
                   xs, ys, lut=None, key_channels=None):
    """RGBA8 output at selected pixels, each computed from scratch."""
    t, kt = _guide(tgt_guide)
    s, ks = _guide(src_guide)
    st, kst = _style(style)
    kc = s.channels if key_channels is None else key_channels
    if lut is None:
        lut = new_lut(kc, key_bits)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    out = np.empty((len(xs), 4), dtype=np.uint8)
    _load().orc_stylize_points(ctypes.byref(t), ctypes.byref(s), ctypes.byref(st), key_bits,
                               kc, _lut_ptr(lut), levels, int(threshold), radius, seed & 0xFFFFFFFF,
                               _ptr(xs), _ptr(ys), len(xs), _ptr(out))
    return out


def lookup_only(tgt_guide, src_guide, style, key_bits, lut=None, key_channels=None):
    """Texture-mapping comparator (§4): C_T[p] = C_S[LUT(G_T[p])]."""
    t, kt = _guide(tgt_guide)
    s, ks = _guide(src_guide)
    st, kst = _style(style)
    kc = s.channels if key_channels is None else key_channels
    if lut is None:
        lut = new_lut(kc, key_bits)
    out = np.empty((t.height, t.width, 4), dtype=np.uint8)
    _load().orc_lookup_only(ctypes.byref(t), ctypes.byref(s), ctypes.byref(st), key_bits, kc,
                            _lut_ptr(lut), _ptr(out))
    return out

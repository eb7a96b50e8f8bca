"""GB300 (sm_103a) StyleBlit: Python binding of the C ABI in include/styleblit.h.

StyleBlit (Sýkora, Jamriška, Lu, Shechtman, EGSR 2018) stylises a target by
copying translated chunks of a style exemplar, chosen per pixel by walking a
hierarchy of jittered seeds (Algorithm 2) and blended by voting (§3.2).

This module only marshals arguments: torch tensors supply device memory and
the current CUDA stream, and every step of the method runs in the CUDA
library `libstyleblit.so`.  There is no CPU fallback: importing the binding
raises if the library cannot be loaded.

Tensor layouts (all on one CUDA device, C-contiguous rows):
  guide  uint8 [H, W, C] (C = 1..4) or int16/uint16-bits [H, W, C] (C = 1..2)
  style  uint8 [H, W, 4] (RGBA8)
  assign int32 [H, W] holding x | y << 16 (uint32 bit pattern)
  level  uint8 [H, W]
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import _build

__all__ = ["StyleBlitError", "Lut", "build_lut", "assign_chunks", "blend", "stylize",
           "stylize_batch", "autotune_batch", "BatchFrame", "lookup_only", "lookup_only_batch",
           "stylize_host",
           "stylize_batch_host",
           "library_path", "load_library",
           "EXPORTED_SYMBOLS", "version", "MAX_BATCH"]

MAX_BATCH = 128

SB_OK = 0
_STATUS = {0: "SB_OK", -1: "SB_ERR_INVALID_ARG", -2: "SB_ERR_UNSUPPORTED", -3: "SB_ERR_CUDA",
           -4: "SB_ERR_OOM", -5: "SB_ERR_TIMEOUT"}

EXPORTED_SYMBOLS = ["sb_build_lut", "sb_build_lut_keyed", "sb_build_lut_noalloc", "sb_lut_destroy", "sb_lut_info",
                    "sb_assign_chunks", "sb_blend", "sb_stylize", "sb_stylize_batch",
                    "sb_stylize_batch_sched", "sb_autotune_batch", "sb_lookup_only",
                    "sb_lookup_only_batch",
                    "sb_status_string", "sb_last_error", "sb_version"]


class StyleBlitError(RuntimeError):
    def __init__(self, fn: str, status: int, message: str):
        super().__init__(f"{fn} failed with {_STATUS.get(status, status)}: {message}")
        self.status = status


class _Guide(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("channels", ctypes.c_int32),
                ("bits", ctypes.c_int32), ("row_stride", ctypes.c_int64)]


class _Rgba8(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("row_stride", ctypes.c_int64)]


class _Schedule(ctypes.Structure):
    _fields_ = [("persistent", ctypes.c_int32), ("largest_first", ctypes.c_int32),
                ("interleave_rows", ctypes.c_int32), ("tile_rows", ctypes.c_int32)]


class _Frame(ctypes.Structure):
    _fields_ = [("tgt_guide", _Guide), ("lut", ctypes.c_void_p), ("src_style", _Rgba8),
                ("levels", ctypes.c_int32), ("threshold", ctypes.c_uint64),
                ("seed", ctypes.c_uint32), ("rgba8_out", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Loads libstyleblit.so (building it with nvcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise ImportError(f"StyleBlit CUDA library not found at {path}")
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER
        vp, i32, i64, u32, u64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                  ctypes.c_uint32, ctypes.c_uint64)
        sigs = {
            "sb_build_lut": (ctypes.c_int, [P(_Guide), i32, P(vp), vp]),
            "sb_build_lut_noalloc": (ctypes.c_int, [P(_Guide), i32, vp, vp]),
            "sb_build_lut_keyed": (ctypes.c_int, [P(_Guide), i32, i32, P(vp), vp]),
            "sb_lut_destroy": (ctypes.c_int, [vp]),
            "sb_lut_info": (ctypes.c_int, [vp, P(vp), P(i64), P(i32), P(i32), P(i32), P(i32),
                                           P(i32), P(i32)]),
            "sb_assign_chunks": (ctypes.c_int, [P(_Guide), P(_Guide), vp, i32, u64, u32, vp, vp,
                                                vp]),
            "sb_blend": (ctypes.c_int, [vp, i32, i32, P(_Rgba8), i32, vp, vp, vp]),
            "sb_stylize": (ctypes.c_int, [P(_Guide), P(_Guide), P(_Rgba8), vp, i32, u64, i32,
                                          u32, vp, vp]),
            "sb_stylize_batch": (ctypes.c_int, [P(_Frame), i32, i32, vp]),
            "sb_lookup_only_batch": (ctypes.c_int, [P(_Frame), i32, vp]),
            "sb_stylize_batch_sched": (ctypes.c_int, [P(_Frame), i32, i32, P(_Schedule), vp]),
            "sb_autotune_batch": (ctypes.c_int, [P(_Frame), i32, i32, i32, P(_Schedule),
                                                 P(ctypes.c_float), vp]),
            "sb_lookup_only": (ctypes.c_int, [P(_Guide), P(_Guide), P(_Rgba8), vp, vp, vp]),
            "sb_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "sb_last_error": (ctypes.c_char_p, []),
            "sb_version": (i32, []),
        }
        for name, (res, args) in sigs.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(fn: str, status: int):
    if status != SB_OK:
        msg = load_library().sb_last_error()
        raise StyleBlitError(fn, status, msg.decode() if msg else "")


def version() -> int:
    return int(load_library().sb_version())


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _guide(t: torch.Tensor, name: str) -> _Guide:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dim() == 2:
        t = t.unsqueeze(-1)
    if t.dim() != 3:
        raise ValueError(f"{name} must be [H, W, C]")
    h, w, c = t.shape
    # strides of dimensions of size <= 1 carry no layout information
    if t.numel() and ((c > 1 and t.stride(2) != 1) or (w > 1 and t.stride(1) != c)):
        raise ValueError(f"{name} must be [H, W, C] with contiguous pixels")
    if t.dtype == torch.uint8:
        bits = 8
    elif t.dtype in (torch.int16, torch.uint16):
        bits = 16
    else:
        raise TypeError(f"{name}: dtype must be uint8 or (u)int16, got {t.dtype}")
    row = w * c * t.element_size()
    stride = t.stride(0) * t.element_size() if (h > 1 and t.numel()) else row
    return _Guide(t.data_ptr(), w, h, c, bits, stride)


def _style(t: torch.Tensor, name: str = "style") -> _Rgba8:
    if not t.is_cuda or t.dtype != torch.uint8 or t.dim() != 3 or t.shape[2] != 4:
        raise ValueError(f"{name} must be a CUDA uint8 tensor [H, W, 4]")
    h, w, _ = t.shape
    if t.stride(2) != 1 or (w > 1 and t.stride(1) != 4):
        raise ValueError(f"{name} must have contiguous RGBA pixels")
    return _Rgba8(t.data_ptr(), w, h, t.stride(0) if h > 1 else 4 * w)


class _DeviceArray:
    """A library-owned int32 device array exposed through __cuda_array_interface__."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<i4", "data": (ptr, False),
                                         "version": 2}


class Lut:
    """A device-resident guide look-up table (Section 3.1), owned by the library."""

    def __init__(self, handle: int, src_shape, device: torch.device):
        self._h = ctypes.c_void_p(handle)
        self.src_shape = tuple(src_shape)
        self.device = device
        info = self.info()
        self.n_entries = info["n_entries"]
        self.key_bits = info["key_bits"]

    @property
    def handle(self) -> ctypes.c_void_p:
        if not self._h:
            raise ValueError("Lut has been destroyed")
        return self._h

    def info(self) -> dict:
        e = ctypes.c_void_p()
        n = ctypes.c_int64()
        c, b, k, kc, w, h = (ctypes.c_int32() for _ in range(6))
        _check("sb_lut_info", load_library().sb_lut_info(
            self.handle, ctypes.byref(e), ctypes.byref(n), ctypes.byref(c), ctypes.byref(b),
            ctypes.byref(k), ctypes.byref(kc), ctypes.byref(w), ctypes.byref(h)))
        return dict(entries_ptr=e.value, n_entries=n.value, channels=c.value, bits=b.value,
                    key_bits=k.value, key_channels=kc.value, src_width=w.value,
                    src_height=h.value)

    def entries(self) -> torch.Tensor:
        """A copy of the table (int32 bit patterns of x | y << 16), ordered on
        the current stream after the work that built it.  Keys wider than 24
        bits have a search index instead of a table (ValueError here)."""
        info = self.info()
        if not info["entries_ptr"]:
            raise ValueError("this object holds a search index, not a table (key wider than 24 bits)")
        view = torch.as_tensor(_DeviceArray(info["entries_ptr"], info["n_entries"]),
                               device=self.device)
        return view.clone()

    def destroy(self):
        if self._h:
            torch.cuda.synchronize(self.device)
            _check("sb_lut_destroy", load_library().sb_lut_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            if self._h:
                self.destroy()
        except Exception:
            pass


def build_lut(src_guide: torch.Tensor, key_bits: int, stream=None, key_channels=None) -> Lut:
    """Guide table (Section 3.1) keyed on every channel, or on the first
    key_channels (extra channels then only enter the acceptance distance)."""
    lib = load_library()
    g = _guide(src_guide, "src_guide")
    h = ctypes.c_void_p()
    kc = g.channels if key_channels is None else key_channels
    _check("sb_build_lut_keyed", lib.sb_build_lut_keyed(ctypes.byref(g), key_bits, kc,
                                                        ctypes.byref(h), _stream(stream)))
    return Lut(h.value, src_guide.shape, src_guide.device)


def assign_chunks(tgt_guide, src_guide, lut: Lut, levels: int, threshold: int, seed: int,
                  with_level: bool = True, out=None, level_out=None, stream=None):
    """Chunk assignment A (int32 [H, W], x | y << 16) and optionally the level map."""
    lib = load_library()
    t, s = _guide(tgt_guide, "tgt_guide"), _guide(src_guide, "src_guide")
    H, W = tgt_guide.shape[:2]
    if out is None:
        out = torch.empty((H, W), dtype=torch.int32, device=tgt_guide.device)
    if with_level and level_out is None:
        level_out = torch.empty((H, W), dtype=torch.uint8, device=tgt_guide.device)
    _check("sb_assign_chunks", lib.sb_assign_chunks(
        ctypes.byref(t), ctypes.byref(s), lut.handle, levels, int(threshold),
        seed & 0xFFFFFFFF, out.data_ptr(), level_out.data_ptr() if with_level else None,
        _stream(stream)))
    return (out, level_out) if with_level else out


def blend(assign: torch.Tensor, style: torch.Tensor, radius: int, f32: bool = False, out=None,
          stream=None):
    """Voting step: RGBA8 [H, W, 4] (uint8) or float32 [H, W, 4] in [0, 1]."""
    lib = load_library()
    if assign.dtype != torch.int32 or not assign.is_contiguous() or assign.dim() != 2:
        raise ValueError("assign must be a contiguous int32 [H, W] tensor")
    H, W = assign.shape
    st = _style(style)
    if out is None:
        out = torch.empty((H, W, 4), dtype=torch.float32 if f32 else torch.uint8,
                          device=assign.device)
    _check("sb_blend", lib.sb_blend(assign.data_ptr(), W, H, ctypes.byref(st), radius,
                                    None if f32 else out.data_ptr(),
                                    out.data_ptr() if f32 else None, _stream(stream)))
    return out


def stylize(tgt_guide, src_guide, style, lut: Lut, levels: int, threshold: int, radius: int,
            seed: int, out=None, stream=None):
    """Fused assignment + vote: RGBA8 [H, W, 4] uint8 on the device."""
    lib = load_library()
    t, s = _guide(tgt_guide, "tgt_guide"), _guide(src_guide, "src_guide")
    st = _style(style)
    H, W = tgt_guide.shape[:2]
    if out is None:
        out = torch.empty((H, W, 4), dtype=torch.uint8, device=tgt_guide.device)
    _check("sb_stylize", lib.sb_stylize(ctypes.byref(t), ctypes.byref(s), ctypes.byref(st),
                                        lut.handle, levels, int(threshold), radius,
                                        seed & 0xFFFFFFFF, out.data_ptr(), _stream(stream)))
    return out


def lookup_only(tgt_guide, src_guide, style, lut: "Lut", out=None, stream=None):
    """Texture-mapping comparator (Section 4): C_T[p] = C_S[LUT(G_T[p])]."""
    lib = load_library()
    t, s = _guide(tgt_guide, "tgt_guide"), _guide(src_guide, "src_guide")
    st = _style(style)
    H, W = tgt_guide.shape[:2]
    if out is None:
        out = torch.empty((H, W, 4), dtype=torch.uint8, device=tgt_guide.device)
    _check("sb_lookup_only", lib.sb_lookup_only(ctypes.byref(t), ctypes.byref(s),
                                                ctypes.byref(st), lut.handle, out.data_ptr(),
                                                _stream(stream)))
    return out


class BatchFrame:
    """One frame of stylize_batch: its target guide, exemplar (table + style),
    level count, threshold, seed and output (allocated when None)."""

    def __init__(self, tgt_guide, lut: "Lut", style, levels: int, threshold: int, seed: int,
                 out=None):
        self.tgt_guide, self.lut, self.style = tgt_guide, lut, style
        self.levels, self.threshold, self.seed = levels, threshold, seed
        if out is None:
            H, W = tgt_guide.shape[:2]
            out = torch.empty((H, W, 4), dtype=torch.uint8, device=tgt_guide.device)
        self.out = out


def _frames_array(frames):
    arr = (_Frame * max(1, len(frames)))()
    for k, f in enumerate(frames):
        arr[k] = _Frame(_guide(f.tgt_guide, f"frames[{k}].tgt_guide"), f.lut.handle,
                        _style(f.style, f"frames[{k}].style"), f.levels, int(f.threshold),
                        f.seed & 0xFFFFFFFF, f.out.data_ptr())
    return arr


def stylize_batch(frames, radius: int, stream=None, schedule: dict | None = None):
    """Stylises up to MAX_BATCH frames (BatchFrame) in one launch; returns their
    outputs.  Frames share the guide format and the blend radius.  `schedule`
    ({"persistent": 0/1, "largest_first": 0/1, "interleave_rows": 0/1,
    "tile_rows": 0/16/32/64}, e.g. from autotune_batch; missing keys are 0)
    picks the launch form; every schedule gives the same pixels."""
    lib = load_library()
    frames = list(frames)
    arr = _frames_array(frames)
    if schedule is None:
        _check("sb_stylize_batch", lib.sb_stylize_batch(arr, len(frames), radius, _stream(stream)))
    else:
        sc = _Schedule(int(schedule.get("persistent", 0)), int(schedule.get("largest_first", 0)),
                       int(schedule.get("interleave_rows", 0)), int(schedule.get("tile_rows", 0)))
        _check("sb_stylize_batch_sched",
               lib.sb_stylize_batch_sched(arr, len(frames), radius, ctypes.byref(sc),
                                          _stream(stream)))
    return [f.out for f in frames]


def lookup_only_batch(frames, stream=None):
    """The lookup-only comparator (Section 4) for up to MAX_BATCH frames
    (BatchFrame; their levels, threshold and seed are ignored) in one launch;
    returns their outputs.  Frames share the guide format."""
    lib = load_library()
    frames = list(frames)
    arr = _frames_array(frames)
    _check("sb_lookup_only_batch", lib.sb_lookup_only_batch(arr, len(frames), _stream(stream)))
    return [f.out for f in frames]


def autotune_batch(frames, radius: int, reps: int = 5, stream=None):
    """Times the launch schedules on this batch (writing its outputs) and
    returns (fastest schedule as a dict, its mean ms per batch)."""
    lib = load_library()
    frames = list(frames)
    arr = _frames_array(frames)
    best, ms = _Schedule(), ctypes.c_float()
    _check("sb_autotune_batch", lib.sb_autotune_batch(arr, len(frames), radius, reps,
                                                      ctypes.byref(best), ctypes.byref(ms),
                                                      _stream(stream)))
    return {"persistent": best.persistent, "largest_first": best.largest_first,
            "interleave_rows": best.interleave_rows, "tile_rows": best.tile_rows}, ms.value


def stylize_batch_host(guides_host, luts, styles, levels, thresholds, seeds, radius: int,
                       outs_host, group: int = 6, streams=None, staging: dict | None = None,
                       schedule: dict | None = None):
    """Stylises frames held in pinned host memory into pinned host memory.

    Frames go in groups of `group`: the group's guides are copied in, one
    sb_stylize_batch launch stylises them, the RGBA8 results are copied out,
    all enqueued on one of `streams` (consecutive groups on consecutive streams,
    so one group's copies overlap the neighbouring groups' kernels).  `luts`,
    `styles`, `levels`, `thresholds` and `seeds` are per frame (a single value
    applies to every frame).  `staging` caches the device buffers between calls;
    `schedule` is passed to stylize_batch.  Returns `outs_host`; the caller
    synchronises the streams before reading it."""
    n = len(guides_host)
    per = lambda v: v if isinstance(v, (list, tuple)) else [v] * n
    luts, styles, levels, thresholds, seeds = map(per, (luts, styles, levels, thresholds, seeds))
    dev = styles[0].device
    streams = list(streams) if streams else [torch.cuda.current_stream(dev)]
    staging = {} if staging is None else staging
    for g0 in range(0, n, group):
        ks = range(g0, min(n, g0 + group))
        stream = streams[(g0 // group) % len(streams)]
        with torch.cuda.stream(stream):
            frames = []
            for k in ks:
                key = (k, tuple(guides_host[k].shape), guides_host[k].dtype)
                if key not in staging:
                    staging[key] = (torch.empty(guides_host[k].shape, dtype=guides_host[k].dtype,
                                                device=dev),
                                    torch.empty(outs_host[k].shape, dtype=torch.uint8, device=dev))
                g, o = staging[key]
                g.copy_(guides_host[k], non_blocking=True)
                frames.append(BatchFrame(g, luts[k], styles[k], levels[k], thresholds[k], seeds[k],
                                         out=o))
            stylize_batch(frames, radius, stream=stream, schedule=schedule)
            for k, f in zip(ks, frames):
                outs_host[k].copy_(f.out, non_blocking=True)
    return outs_host


def stylize_host(tgt_guide_host: torch.Tensor, src_guide, style, lut: Lut, levels: int,
                 threshold: int, radius: int, seed: int, out_host: torch.Tensor,
                 staging: dict | None = None, stream=None):
    """Stylises a frame held in (pinned) host memory into host memory: the guide
    is copied in, sb_stylize runs, the RGBA8 result is copied out, all enqueued
    on `stream`.  `staging` caches the device buffers between calls."""
    if stream is not None:
        with torch.cuda.stream(stream):
            return stylize_host(tgt_guide_host, src_guide, style, lut, levels, threshold,
                                radius, seed, out_host, staging)
    dev = src_guide.device
    staging = {} if staging is None else staging
    key = (tuple(tgt_guide_host.shape), tgt_guide_host.dtype)
    if staging.get("key") != key:
        staging["key"] = key
        staging["g"] = torch.empty(tgt_guide_host.shape, dtype=tgt_guide_host.dtype, device=dev)
        staging["o"] = torch.empty(out_host.shape, dtype=torch.uint8, device=dev)
    g, o = staging["g"], staging["o"]
    g.copy_(tgt_guide_host, non_blocking=True)
    stylize(g, src_guide, style, lut, levels, threshold, radius, seed, out=o)
    out_host.copy_(o, non_blocking=True)
    return out_host

"""The C ABI library builds, loads without a GPU, exports every function that
include/styleblit.h declares, and rejects invalid arguments on the host before
touching the device (these paths never call CUDA)."""
import ctypes
import os
import re

import pytest

import paper_1807_03249_gb300 as sb

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "styleblit.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"SB_API\s+[\w\s\*]+?\b(sb_\w+)\s*\(", text)))


def test_header_declares_the_expected_entry_points():
    names = _declared()
    for n in ["sb_build_lut", "sb_assign_chunks", "sb_blend", "sb_stylize"]:
        assert n in names
    assert set(names) == set(sb.EXPORTED_SYMBOLS)


def test_library_exports_every_declared_symbol():
    lib = sb.load_library()
    for name in _declared():
        assert hasattr(lib, name), name
    assert sb.version() == 10000
    assert lib.sb_status_string(0) == b"SB_OK"
    assert b"INVALID" in lib.sb_status_string(-1)


def _guide(w, h, c, bits, ptr=0x1000, stride=None):
    if stride is None:
        stride = w * c * bits // 8
    return sb._Guide(ptr, w, h, c, bits, stride)


def _call_stylize(tgt, src, radius=2, levels=4, lut=None, style_wh=None):
    lib = sb.load_library()
    sw, sh = style_wh or (src.width, src.height)
    st = sb._Rgba8(0x2000, sw, sh, 4 * sw)
    return lib.sb_stylize(ctypes.byref(tgt), ctypes.byref(src), ctypes.byref(st), lut, levels,
                          300, radius, 0, 0x3000, None)


@pytest.mark.parametrize("tgt,src,status", [
    (_guide(64, 64, 3, 12), _guide(64, 64, 3, 12), -1),      # bits not 8/16
    (_guide(64, 64, 3, 16), _guide(64, 64, 3, 16), -2),      # 16-bit x 3 unsupported
    (_guide(64, 64, 5, 8), _guide(64, 64, 5, 8), -1),        # 5 channels
    (_guide(64, 64, 3, 8), _guide(40000, 8, 3, 8), -1),      # source too wide
    (_guide(65536, 2, 3, 8), _guide(64, 64, 3, 8), -1),      # target too wide
    (_guide(64, 64, 3, 8), _guide(0, 8, 3, 8), -1),          # empty source
    (_guide(64, 64, 3, 8), _guide(64, 64, 2, 8), -1),        # channel mismatch
    (_guide(64, 64, 3, 8, stride=10), _guide(64, 64, 3, 8), -1),   # short stride
    (_guide(64, 64, 4, 8, ptr=0x1002), _guide(64, 64, 4, 8), -1),  # misaligned
    (_guide(64, 64, 3, 8), _guide(64, 64, 3, 8), -1),        # NULL lut
])
def test_invalid_frame_arguments_are_rejected_on_the_host(tgt, src, status):
    assert _call_stylize(tgt, src) == status
    assert sb.load_library().sb_last_error() != b""


def test_invalid_blend_and_lut_arguments_are_rejected_on_the_host():
    lib = sb.load_library()
    st = sb._Rgba8(0x2000, 16, 16, 64)
    # neither output
    assert lib.sb_blend(0x1000, 8, 8, ctypes.byref(st), 1, None, None, None) == -1
    # both outputs
    assert lib.sb_blend(0x1000, 8, 8, ctypes.byref(st), 1, 0x3000, 0x4000, None) == -1
    # radius out of range
    assert lib.sb_blend(0x1000, 8, 8, ctypes.byref(st), 16, 0x3000, None, None) == -1
    # bad style stride
    bad = sb._Rgba8(0x2000, 16, 16, 60)
    assert lib.sb_blend(0x1000, 8, 8, ctypes.byref(bad), 1, 0x3000, None, None) == -1
    h = ctypes.c_void_p()
    g = _guide(32, 32, 3, 8)
    assert lib.sb_build_lut(ctypes.byref(g), 0, ctypes.byref(h), None) == -1
    assert lib.sb_build_lut(ctypes.byref(g), 9, ctypes.byref(h), None) == -1
    g4 = _guide(32, 32, 4, 8)
    assert lib.sb_build_lut_keyed(ctypes.byref(g4), 7, 5, ctypes.byref(h), None) == -1  # 5 > 4 channels
    assert lib.sb_build_lut_keyed(ctypes.byref(g4), 7, 0, ctypes.byref(h), None) == -1  # no channel
    assert lib.sb_build_lut(None, 6, ctypes.byref(h), None) == -1
    assert h.value is None
    assert lib.sb_lut_destroy(None) == 0


def test_invalid_batch_and_schedule_arguments_are_rejected_on_the_host():
    lib = sb.load_library()
    frames = (sb._Frame * 1)()
    sched = sb._Schedule(1, 1, 0, 0)
    best, ms = sb._Schedule(), ctypes.c_float()
    assert lib.sb_stylize_batch(frames, 129, 2, None) == -1            # too many frames
    assert lib.sb_stylize_batch(None, 1, 2, None) == -1                # NULL frames
    assert lib.sb_stylize_batch_sched(frames, 1, 16, ctypes.byref(sched), None) == -1  # radius
    bad_rows = sb._Schedule(0, 0, 0, 48)
    assert lib.sb_stylize_batch_sched(frames, 1, 2, ctypes.byref(bad_rows), None) == -1
    assert b"tile_rows" in lib.sb_last_error()
    tall = sb._Schedule(0, 0, 0, 64)
    assert lib.sb_stylize_batch_sched(frames, 1, 9, ctypes.byref(tall), None) == -1  # r > 7
    assert lib.sb_stylize_batch_sched(frames, -1, 2, None, None) == -1
    assert lib.sb_stylize_batch_sched(frames, 0, 2, None, None) == 0   # empty batch: no-op
    assert lib.sb_autotune_batch(frames, 1, 2, 3, None, ctypes.byref(ms), None) == -1  # no best
    assert lib.sb_autotune_batch(frames, 1, 2, 0, ctypes.byref(best), None, None) == -1  # reps
    assert b"reps" in lib.sb_last_error()
    assert lib.sb_lookup_only_batch(frames, 129, None) == -1           # too many frames
    assert lib.sb_lookup_only_batch(None, 1, None) == -1               # NULL frames
    assert lib.sb_lookup_only_batch(frames, -1, None) == -1
    assert lib.sb_lookup_only_batch(frames, 0, None) == 0              # empty batch: no-op
    assert lib.sb_lookup_only_batch(frames, 1, None) == -1             # frame 0 has no guide
    assert b"frames[0]" in lib.sb_last_error()


def test_style_too_large_for_32_bit_offsets_is_rejected():
    """The kernels address the style with 32-bit pixel offsets: height times
    row stride must stay below 2^31 pixels."""
    lib = sb.load_library()
    st = sb._Rgba8(0x2000, 64, 64, 4 * (1 << 26))  # 64 rows of 2^26 pixels
    assert lib.sb_blend(0x1000, 8, 8, ctypes.byref(st), 1, 0x3000, None, None) == -1
    assert b"2^33" in lib.sb_last_error()

"""sb_build_lut_noalloc: the guide table built into caller-owned memory with
no device allocation, for callers that cannot allocate (e.g. a host
application whose pool allocator owns the GPU's memory, or a frame loop that
must not call cudaMalloc).  Its entries must equal the oracle's table (whole
table where the oracle's brute force is quick, sampled bins otherwise) and
the entries of sb_build_lut.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  It calls the entry point
through the C ABI (ctypes), several times in a row on different sources, so
later calls also show that the shared fixed scratch left by an earlier call
does not leak into the result.  Two sources sit at the edge of the fixed
scratch: exactly 65536 tiles of 16 x 16 pixels, and the largest super-tile
count a source with at most 65536 tiles can have.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1807_03249_gb300 as sb
import synth

pytestmark = pytest.mark.gpu


def _to_dev(a, dev):
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _noalloc(lib, g: torch.Tensor, key_bits: int) -> torch.Tensor:
    desc = sb._guide(g, "src_guide")
    out = torch.full((1 << (desc.channels * key_bits),), -1, dtype=torch.int32, device=g.device)
    stream = torch.cuda.current_stream(g.device).cuda_stream
    status = lib.sb_build_lut_noalloc(ctypes.byref(desc), key_bits, out.data_ptr(), stream)
    assert status == 0, lib.sb_last_error()
    return out


def _edge_guide(seed: int, h: int, w: int) -> np.ndarray:
    """A one-channel 8-bit guide of smooth integer values with a few repeats."""
    return synth.smooth_integer_guide(seed, h, w, 1, step=3)


# (source, key_bits, whole table against the oracle?)
def _cases():
    return [
        (synth.sphere_normals(96), 5, True),
        (synth.identity_uv_guide(384, 512), 9, False),
        (synth.random_guide(3, 77, 131, 2, bits=8, low=20, high=90), 7, True),
        (_edge_guide(41, 4096, 4096), 6, True),    # 256 x 256 = 65536 tiles
        (_edge_guide(42, 31760, 528), 6, True),    # 1985 x 33 tiles, 497 x 9 = 4473 super-tiles
    ]


def test_noalloc_table_equals_oracle_and_allocating_build_in_a_row(cuda_device):
    lib = sb.load_library()
    rng = np.random.default_rng(17)
    for k, (src, key_bits, whole) in enumerate(_cases()):
        g = _to_dev(src, cuda_device)
        got = _noalloc(lib, g, key_bits)
        ref = sb.build_lut(g, key_bits).entries()
        torch.cuda.synchronize()
        assert torch.equal(got, ref), f"case {k}: differs from sb_build_lut"
        tab = got.cpu().numpy().view(np.uint32)
        if whole:
            assert np.array_equal(tab, oracle.build_lut(src, key_bits)), f"case {k}"
        else:
            idx = np.concatenate([rng.integers(0, tab.shape[0], 10000), [0, tab.shape[0] - 1]])
            assert np.array_equal(tab[idx], oracle.lut_entries(src, key_bits, idx)), f"case {k}"


def test_noalloc_rejects_sources_beyond_the_fixed_scratch(cuda_device):
    lib = sb.load_library()
    out = torch.empty(1 << 18, dtype=torch.int32, device=cuda_device)
    # 257 x 256 tiles > 65536; then 33 x 1986 tiles (65538 > 65536)
    for w, h in ((4097, 4096), (528, 31776)):
        desc = sb._Guide(0x1000, w, h, 3, 8, w * 3)
        status = lib.sb_build_lut_noalloc(ctypes.byref(desc), 6, out.data_ptr(), None)
        assert status == -1
        assert b"too large" in lib.sb_last_error()

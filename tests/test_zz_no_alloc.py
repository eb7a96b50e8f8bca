"""sb_build_lut_noalloc: the guide table built into caller-owned memory with
no device allocation, for callers that cannot allocate (e.g. a host
application whose pool allocator owns the GPU's memory, or a frame loop that
must not call cudaMalloc).  It must give exactly the entries of sb_build_lut.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  It calls the entry point
through the C ABI (ctypes), twice in a row on different sources, so the
second call also shows that the shared fixed scratch left by the first call
does not leak into the result.
"""
import ctypes

import numpy as np
import pytest
import torch

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


def test_noalloc_table_equals_allocating_build_twice_in_a_row(cuda_device):
    lib = sb.load_library()
    cases = [(synth.sphere_normals(256), 6),
             (synth.identity_uv_guide(384, 512), 9),
             (synth.random_guide(3, 77, 131, 2, bits=8, low=20, high=90), 7)]
    for src, key_bits in cases:
        g = _to_dev(src, cuda_device)
        got = _noalloc(lib, g, key_bits)
        ref = sb.build_lut(g, key_bits).entries()
        torch.cuda.synchronize()
        assert torch.equal(got, ref)


def test_noalloc_rejects_sources_beyond_the_fixed_scratch(cuda_device):
    lib = sb.load_library()
    desc = sb._Guide(0x1000, 4097, 4096, 3, 8, 4097 * 3)  # 257 x 256 tiles > 65536
    out = torch.empty(1 << 18, dtype=torch.int32, device=cuda_device)
    status = lib.sb_build_lut_noalloc(ctypes.byref(desc), 6, out.data_ptr(), None)
    assert status == -1
    assert b"too large" in lib.sb_last_error()

"""Animation on the GPU (Section 3.3): every frame of a sequence stylised in
one launch equals the oracle's stylisation of that frame with the same frame
seed, equals the frame stylised alone, and the sequence shows the flicker
ordering of Section 3.3 (fixed seed coherent, per-frame seeds flicker more)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1807_03249_gb300 as sb
import synth
from paper_1807_03249_gb300.animation import flicker, frame_seed, stylize_sequence
from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu


def test_sequence_matches_oracle_per_frame_and_flicker_ordering(cuda_device):
    ex = synth.normal_exemplar(9, 256, octaves=3, lut_bits=6)
    gs, st = to_dev(ex.guide, cuda_device), to_dev(ex.style, cuda_device)
    lut = sb.build_lut(gs, 6)
    base = synth.bump_normals(78, 270, 480, 16, (8.0, 64.0))
    host = [np.ascontiguousarray(base[:, t:t + 400]) for t in range(0, 16, 2)]
    guides = [to_dev(g, cuda_device) for g in host]
    ref_lut = oracle.new_lut(3, 6)
    res = {}
    for mode in ("static", "per_frame"):
        outs = stylize_sequence(guides, lut, st, 5, 300, 2, 4321, mode)
        torch.cuda.synchronize()
        for t, g in enumerate(host):
            ref, _, _ = oracle.stylize(g, ex.guide, ex.style, 6, 5, 300, 2,
                                       frame_seed(4321, t, mode), lut=ref_lut, n_threads=4)
            assert np.array_equal(outs[t].cpu().numpy(), ref), f"{mode} frame {t}"
        for t in (0, 5):
            single = sb.stylize(guides[t], gs, st, lut, 5, 300, 2, frame_seed(4321, t, mode))
            assert torch.equal(outs[t], single)
        res[mode] = flicker(outs)
    torch.cuda.synchronize()
    assert res["static"] < res["per_frame"]

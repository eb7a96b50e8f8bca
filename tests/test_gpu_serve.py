"""The serving loop: requests of mixed sizes and exemplars, admitted while
others are on the GPU, give exactly the result each gives alone, and that
result equals the oracle's stylisation of the request."""
import numpy as np
import pytest
import torch

import oracle
import paper_1807_03249_gb300 as sb
import synth
from paper_1807_03249_gb300.serve import Request, Server

pytestmark = pytest.mark.gpu


def test_served_results_equal_each_request_alone(cuda_device):
    rng = np.random.default_rng(5)
    srv = Server(cuda_device, radius=2, budget_bytes=0, slots=2, max_batch=4)
    exs = {}
    for k in range(3):
        g = synth.sphere_normals(96 + 32 * k)
        st = synth.value_noise_style(300 + k, g.shape[0], g.shape[1], octaves=3, base_cell=16)
        srv.add_exemplar(k, g, st, key_bits=5)
        exs[k] = (g, st)
    reqs = []
    for i in range(14):
        w, h = int(rng.integers(8, 400)), int(rng.integers(8, 300))
        g = torch.from_numpy(synth.bump_normals(700 + i, h, w, 4, (5.0, 40.0))).pin_memory()
        reqs.append(Request(i, 0.0, i % 3, g, int(rng.integers(2, 7)), int(rng.integers(50, 800)),
                            int(rng.integers(0, 2**32))))
    # budget: the two largest requests at once, so admission has to wait at times
    sizes = sorted(srv.device_bytes(r.guide) for r in reqs)
    srv.sched.budget = sizes[-1] + sizes[-2]
    done, wall = srv.run(reqs, real_time=False)
    assert len(done) == len(reqs)
    assert srv.sched.peak_in_use <= srv.sched.budget and srv.sched.in_use == 0
    ref_luts = {k: oracle.new_lut(3, 5) for k in exs}
    for r in reqs:
        gd, sd, lut = srv.exemplars[r.exemplar]
        alone = sb.stylize(r.guide.to(cuda_device), gd, sd, lut, r.levels, r.threshold, 2, r.seed)
        torch.cuda.synchronize()
        assert torch.equal(r.out, alone.cpu()), f"request {r.rid}"
        g, stl = exs[r.exemplar]
        ref, _, _ = oracle.stylize(r.guide.numpy(), g, stl, 5, r.levels, r.threshold, 2, r.seed,
                                   lut=ref_luts[r.exemplar], n_threads=4)
        assert np.array_equal(r.out.numpy(), ref), f"request {r.rid} vs oracle"
        assert r.done >= r.admitted >= r.arrival


def test_reserved_server_allocates_no_device_memory_while_serving(cuda_device):
    """After Server.reserve, serving a stream of mixed sizes makes no device
    allocation (guides and outputs live in the slot arenas) and every result
    still equals the request alone."""
    rng = np.random.default_rng(9)
    srv = Server(cuda_device, radius=2, budget_bytes=1 << 30, slots=3, max_batch=4)
    g = synth.sphere_normals(128)
    st = synth.value_noise_style(9, 128, 128, octaves=3, base_cell=16)
    srv.add_exemplar(0, g, st, key_bits=5)
    reqs = []
    for i in range(24):
        w, h = int(rng.integers(1, 500)), int(rng.integers(1, 300))
        gi = torch.from_numpy(synth.bump_normals(900 + i, h, w, 4, (5.0, 40.0))).pin_memory()
        reqs.append(Request(i, 0.0, 0, gi, 5, 300, int(rng.integers(0, 2**32)),
                            out=torch.empty((h, w, 4), dtype=torch.uint8).pin_memory()))
    srv.reserve(sum(sorted(srv.device_bytes(r.guide) for r in reqs)[-4:]))
    torch.cuda.synchronize()
    before = torch.cuda.memory_stats(cuda_device)["allocation.all.allocated"]
    done, _ = srv.run(reqs, real_time=False)
    after = torch.cuda.memory_stats(cuda_device)["allocation.all.allocated"]
    assert len(done) == len(reqs) and after == before
    _, sd, lut = srv.exemplars[0]
    gd = srv.exemplars[0][0]
    ref_lut = oracle.new_lut(3, 5)
    for r in reqs:
        alone = sb.stylize(r.guide.to(cuda_device), gd, sd, lut, 5, 300, 2, r.seed)
        torch.cuda.synchronize()
        assert torch.equal(r.out, alone.cpu()), f"request {r.rid}"
        ref, _, _ = oracle.stylize(r.guide.numpy(), g, st, 5, 5, 300, 2, r.seed, lut=ref_lut,
                                   n_threads=4)
        assert np.array_equal(r.out.numpy(), ref), f"request {r.rid} vs oracle"

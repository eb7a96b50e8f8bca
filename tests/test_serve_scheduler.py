"""Admission rules of the serving loop's scheduler (no GPU): arrival order,
slots, byte budget (never exceeded), group size, oversized requests refused."""
import numpy as np
import pytest

from paper_1807_03249_gb300.serve import Request, Scheduler, latency_summary


def _req(rid, nbytes, arrival=0.0):
    r = Request(rid, arrival, 0, np.zeros((2, 3, 3), np.uint8), 1, 0, 0)
    r.nbytes = nbytes
    return r


def test_fifo_groups_respect_slots_budget_and_batch_size():
    s = Scheduler(budget_bytes=100, slots=2, max_batch=3)
    for i, b in enumerate([30, 30, 30, 30, 50, 10]):
        s.submit(_req(i, b))
    slot, g = s.next_group()
    assert [r.rid for r in g] == [0, 1, 2] and s.in_use == 90      # max_batch 3
    assert s.next_group() is None                                  # head (30) does not fit
    s.finish(slot, g)
    slot2, g2 = s.next_group()
    assert [r.rid for r in g2] == [3, 4, 5]                        # 30 + 50 + 10 = 90 fits
    assert s.in_use == 90 and s.peak_in_use <= s.budget


def test_slots_limit_concurrent_groups_and_budget_never_exceeded():
    rng = np.random.default_rng(0)
    s = Scheduler(budget_bytes=1000, slots=3, max_batch=4)
    for i in range(200):
        s.submit(_req(i, int(rng.integers(1, 400))))
    inflight, order = [], []
    while s.waiting or inflight:
        nxt = s.next_group()
        if nxt is not None:
            inflight.append(nxt)
            assert len(inflight) <= 3
            assert s.in_use <= 1000
            order.extend(r.rid for r in nxt[1])
            continue
        slot, g = inflight.pop(0)
        s.finish(slot, g)
    assert order == list(range(200))        # arrival order kept
    assert s.in_use == 0 and s.peak_in_use <= 1000 and sorted(s.free_slots) == [0, 1, 2]


def test_oversized_request_is_refused():
    s = Scheduler(budget_bytes=10, slots=1, max_batch=1)
    with pytest.raises(ValueError):
        s.submit(_req(0, 11))


def test_latency_summary():
    reqs = [_req(i, 1, arrival=0.0) for i in range(100)]
    for i, r in enumerate(reqs):
        r.done = (i + 1) * 1e-3
    out = latency_summary(reqs, wall_s=0.1)
    assert out["p50_ms"] == pytest.approx(50.5) and out["p99_ms"] == pytest.approx(99.01)
    assert out["frames_per_s"] == pytest.approx(1000)


def test_slot_arena_carves_aligned_disjoint_views_and_grows_in_steps():
    """A slot's arena (host logic, run here on a CPU tensor): views start on
    256-byte boundaries in carve order without overlapping, have the asked
    dtype and shape, the arena grows only in 64 MiB steps, and an overflowing
    carve is refused."""
    torch = pytest.importorskip("torch")
    from paper_1807_03249_gb300.serve import SlotArena

    a = SlotArena(torch, torch.device("cpu"))
    parts = [((5, 7, 3), torch.uint8), ((5, 7, 4), torch.uint8), ((3, 9, 2), torch.int16),
             ((1, 1, 1), torch.uint8), ((2, 3, 4), torch.uint8)]
    need = sum(SlotArena.aligned(torch.empty(sh, dtype=dt).element_size() * sh[0] * sh[1] * sh[2])
               for sh, dt in parts)
    a.start_group(need)
    assert a.capacity == SlotArena.STEP
    a.buf.zero_()
    views = [a.carve(dt, sh) for sh, dt in parts]
    base = a.buf.data_ptr()
    spans = []
    for v, (sh, dt) in zip(views, parts):
        off = v.data_ptr() - base
        assert off % 256 == 0 and v.is_contiguous() and tuple(v.shape) == sh and v.dtype == dt
        spans.append((off, off + v.numel() * v.element_size()))
    assert all(e1 <= s2 for (_, e1), (s2, _) in zip(spans, spans[1:]))
    views[1].fill_(7)
    assert all(int(v.abs().sum()) == 0 for k, v in enumerate(views) if k != 1)
    # a guide [5, 7, 3] uint8 and its RGBA8 output take 256 + 256 bytes
    assert SlotArena.request_bytes(torch.empty((5, 7, 3), dtype=torch.uint8)) == 512
    buf = a.buf
    a.start_group(10)                       # fits: same buffer, carving restarts
    assert a.buf is buf and a.carve(torch.uint8, (1, 1, 4)).data_ptr() == base
    a.start_group(SlotArena.STEP + 1)       # two steps
    assert a.capacity == 2 * SlotArena.STEP and a.buf is not buf
    with pytest.raises(ValueError):
        a.carve(torch.uint8, (a.capacity, 2, 1))

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

"""Host-side tests of the continuous-batching server (no GPU).

A fake executor stands in for the CUDA streams: chunks "finish" after a
number of polls, and their outputs are a deterministic function of the inputs,
so the assembly of split requests and the admission rules can be checked
exactly under a small mocked HBM budget.
"""
import numpy as np
import pytest

from paper_2506_04891_gb300 import serving as S


class FakeExecutor:
    def __init__(self, polls=3):
        self.polls = polls
        self.log = []
        self.max_used = 0

    @staticmethod
    def footprint(n, b):
        return (b << n) * 8 * 3

    def launch(self, req, lo, hi, offset=0):
        self.log.append((req.rid, lo, hi, offset))
        return {"left": self.polls, "req": req, "lo": lo, "hi": hi}

    def done(self, h):
        h["left"] -= 1
        return h["left"] <= 0

    def finish(self, h):
        req, lo, hi = h["req"], h["lo"], h["hi"]
        ez = np.cos(req.x[lo:hi, : req.n])
        dth = req.theta * (hi - lo)
        dx = np.sin(req.x[lo:hi])
        return ez, dth, dx


def _reqs(count=20, seed=3):
    return S.make_requests(count, seed, n_range=(4, 9), b_range=(1, 40))


def test_split_chunks_cover_batch_and_fit():
    ex = FakeExecutor()
    budget = ex.footprint(9, 7)
    sch = S.Scheduler(budget, 4, ex.footprint)
    for r in _reqs():
        chunks = sch.split(r)
        assert chunks[0][0] == 0 and chunks[-1][1] == r.batch
        for (a, b), (c, d) in zip(chunks, chunks[1:]):
            assert b == c
        for a, b in chunks:
            assert ex.footprint(r.n, b - a) <= budget


def test_request_too_large_for_budget_is_rejected():
    ex = FakeExecutor()
    sch = S.Scheduler(ex.footprint(5, 1), 2, ex.footprint)
    r = S.make_requests(1, 0, n_range=(8, 8), b_range=(3, 3))[0]
    with pytest.raises(ValueError):
        sch.split(r)


class BudgetCheckingScheduler(S.Scheduler):
    def admit(self, key, n, b):
        off = super().admit(key, n, b)
        assert self.used <= self.budget
        assert len(self.in_flight) <= self.slots
        # the regions of the chunks in flight are disjoint and inside the arena
        spans = sorted(self.in_flight.values())
        for (o1, s1), (o2, s2) in zip(spans, spans[1:]):
            assert o1 + s1 <= o2
        assert spans[-1][0] + spans[-1][1] <= self.budget
        assert off % S.ALIGN == 0
        self.peak = max(getattr(self, "peak", 0), len(self.in_flight))
        return off


@pytest.mark.parametrize("slots", [1, 2, 5])
def test_mixed_results_equal_direct_computation(slots):
    ex = FakeExecutor(polls=2)
    reqs = _reqs()
    sch = BudgetCheckingScheduler(ex.footprint(9, 24), slots, ex.footprint)
    arrivals = [0.0] * (len(reqs) // 2) + list(np.linspace(0.0, 0.002, len(reqs) - len(reqs) // 2))
    results, stats = S.Server(ex, sch).run(reqs, arrivals)
    assert len(results) == len(reqs)
    for r in reqs:
        res = results[r.rid]
        assert np.array_equal(res.ez, np.cos(r.x[:, : r.n]))
        assert np.array_equal(res.dx, np.sin(r.x))
        assert np.allclose(res.dtheta, r.theta * r.batch)
        assert res.chunks == len(sch.split(r))
        assert res.done >= res.admitted >= res.arrival
    assert sch.used == 0 and not sch.in_flight
    assert sch.free == [(0, sch.budget)]  # every region returned and merged
    if slots > 1:
        assert sch.peak > 1  # work overlapped
    assert stats["p99_ms"] >= stats["p50_ms"] >= 0


def test_poisson_arrivals_are_seeded_and_increasing():
    a = S.poisson_arrivals(100, 50.0, seed=1)
    b = S.poisson_arrivals(100, 50.0, seed=1)
    assert a == b and all(x < y for x, y in zip(a, a[1:]))
    assert abs(np.mean(np.diff(a)) - 1 / 50.0) < 0.01


def test_arena_first_fit_reuses_and_merges_regions():
    sch = S.Scheduler(10 * S.ALIGN, 4, lambda n, b: b * S.ALIGN)
    a = sch.admit("a", 1, 3)
    b = sch.admit("b", 1, 3)
    c = sch.admit("c", 1, 4)
    assert (a, b, c) == (0, 3 * S.ALIGN, 6 * S.ALIGN)
    assert not sch.can_admit(1, 1)
    sch.release("b")
    assert sch.can_admit(1, 3) and not sch.can_admit(1, 4)
    assert sch.admit("d", 1, 2) == 3 * S.ALIGN
    sch.release("a")
    sch.release("c")
    sch.release("d")
    assert sch.free == [(0, 10 * S.ALIGN)] and sch.used == 0

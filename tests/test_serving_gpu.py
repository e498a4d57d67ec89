"""Continuous batching on the GPU: each request's result is the same alone and
in the mix (overlapping streams, a small HBM budget that forces splits), and
matches the oracle on sampled requests."""
import numpy as np
import pytest

from paper_2506_04891_gb300 import serving as S

pytestmark = pytest.mark.gpu


def test_mixed_equals_alone_and_oracle():
    from oracle import qsim_oracle as O
    ex = S.GpuExecutor(slots=4)
    reqs = S.make_requests(24, seed=5, n_range=(8, 14), b_range=(1, 48))
    big = max(reqs, key=lambda r: (r.batch << r.n))
    budget = ex.footprint(big.n, max(1, big.batch // 3))  # the largest request splits into chunks
    mixed, stats = S.Server(ex, S.Scheduler(budget, 4, ex.footprint)).run(
        reqs, S.poisson_arrivals(len(reqs), 400.0, seed=5))
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    assert any(r.chunks > 1 for r in mixed.values())
    for r in S.make_requests(24, seed=5, n_range=(8, 14), b_range=(1, 48)):
        alone, _ = S.Server(ex, S.Scheduler(budget, 1, ex.footprint)).run([r])
        a, m = alone[r.rid], mixed[r.rid]
        assert np.array_equal(a.ez, m.ez)
        assert np.array_equal(a.dx, m.dx)
        assert np.array_equal(a.dtheta, m.dtheta)
    for r in S.make_requests(24, seed=5, n_range=(8, 14), b_range=(1, 48))[:3]:
        layers = S.W.serving_circuit(r.n)
        ez, dth, _, dx = O.adjoint(r.n, layers, r.x, r.theta, r.g)
        m = mixed[r.rid]
        assert np.max(np.abs(m.ez - ez)) < 2e-5
        assert np.max(np.abs(m.dx - dx)) < 2e-5
        assert np.max(np.abs(m.dtheta - dth)) < 2e-5 * r.batch

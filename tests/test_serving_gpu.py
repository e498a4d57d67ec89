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


@pytest.mark.parametrize("name", ["serve20", "serve24"])
def test_serving_large_n_plans_match_oracle_goldens(name):
    """The serving circuit at the stream's largest qubit counts (n = 20: two
    tile passes per rotation layer; n = 24: three, with the RZ layers fused as
    pre / post phases) through GpuExecutor / Server, against the oracle's
    values (tests/golden/<name>.npz, seed 0, B = 2): per-sample <Z>, d theta
    and d x from one-sample requests, the batch request's d theta sum, and 512
    sampled amplitudes of each state from the executor's circuit."""
    import os

    import torch
    G = np.load(os.path.join(os.path.dirname(__file__), "golden", f"{name}.npz"))
    cfg = S.W.WORKLOADS[name]
    n, layers = cfg["n"], cfg["layers"]()
    x, theta, g = S.W.draw_inputs(n, layers, cfg["batch"], seed=0)
    bs = [int(b) for b in G["samples"]]
    ex = S.GpuExecutor(slots=2)
    reqs = [S.Request(k, n, 1, x[b:b + 1], theta, g[b:b + 1]) for k, b in enumerate(bs)]
    reqs.append(S.Request(len(bs), n, len(bs), x[bs], theta, g[bs]))
    big = ex.footprint(n, len(bs))
    res, _ = S.Server(ex, S.Scheduler(2 * big, 2, ex.footprint)).run(reqs)
    dth_ref = dict(zip([int(b) for b in G["dth_samples"]], G["dth"]))
    for k, b in enumerate(bs):
        r = res[k]
        assert np.max(np.abs(r.ez[0] - G["ez"][k])) <= 2e-5, (b, "ez")
        assert np.max(np.abs(r.dx[0] - G["dx"][k])) <= 2e-5, (b, "dx")
        assert np.max(np.abs(r.dtheta - dth_ref[b])) <= 2e-5, (b, "dtheta")
    whole = res[len(bs)]
    assert np.max(np.abs(whole.ez - G["ez"])) <= 2e-5
    assert np.max(np.abs(whole.dx - G["dx"])) <= 2e-5
    assert np.max(np.abs(whole.dtheta - G["dth_sum"])) <= 2e-5 * len(bs)
    c = ex.circuit(n)
    psi, _ = c.forward(torch.tensor(x[bs], device="cuda"), torch.tensor(theta, device="cuda"), ez=False)
    idx = torch.as_tensor(G["psi_idx"], device="cuda")
    got = torch.stack([psi[k][idx[k]] for k in range(len(bs))]).cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(got - G["psi_val"])) <= 2e-5

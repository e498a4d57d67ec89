"""Full-size workloads in the launch configuration the benchmark times.

The CUDA path runs the whole batch; the oracle's values for the listed
samples come from tests/golden/<workload>.npz (written by
tests/golden/make_goldens.py, which calls only the oracle).  Per-sample
d theta is checked by masking the upstream gradient to one sample while the
launch keeps the full batch.  zz26 is also checked against a closed form that
holds at any n (one block: RX, RY, IsingZZ ring, CNOT ring), and so is the
largest register, n = 30.
"""
import os

import numpy as np
import pytest

from paper_2506_04891_gb300 import workloads as W
from tests.gpu_helpers import ABS_C64, REL_C128, check, rel, run_gpu

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    p = os.path.join(GOLD, f"{name}.npz")
    if not os.path.exists(p):
        pytest.skip(f"{p} not generated")
    return np.load(p)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_hea12_full_batch(dtype):
    G = golden("hea12")
    cfg = W.WORKLOADS["hea12"]
    n, layers, B = cfg["n"], cfg["layers"](), cfg["batch"]
    x, theta, g = W.draw_inputs(n, layers, B, seed=0)
    got = run_gpu(n, layers, x, theta, g, dtype=dtype)
    check(dtype, "ez", got["ez"], G["ez"])
    check(dtype, "dx", got["dx"], G["dx"])
    check(dtype, "dtheta", got["dth"], G["dth_sum"], batch_sum=B)
    for k, b in enumerate(G["psi_full_samples"]):
        r = rel(got["psi"][b], G["psi_full"][k])
        assert r <= (REL_C128 if dtype == "c128" else 1e-5), (b, r)


def _sampled(name, dtype="c64"):
    G = golden(name)
    cfg = W.WORKLOADS[name]
    n, layers, B = cfg["n"], cfg["layers"](), cfg["batch"]
    x, theta, g = W.draw_inputs(n, layers, B, seed=0)
    idx = {int(b): G["psi_idx"][k] for k, b in enumerate(G["samples"])}
    got = run_gpu(n, layers, x, theta, g, dtype=dtype, psi=False, psi_idx=idx)
    assert np.allclose(got["norms"], 1.0, atol=1e-5)
    for k, b in enumerate(G["samples"]):
        check(dtype, f"ez[{b}]", got["ez"][b], G["ez"][k])
        check(dtype, f"dx[{b}]", got["dx"][b], G["dx"][k])
        r = rel(got["psi_sel"][int(b)], G["psi_val"][k])
        assert r < 1e-5, (b, r)
    # per-sample d theta: mask the upstream gradient, keep the batch
    del got
    for k, b in enumerate(G["samples"]):
        gm = np.zeros_like(g)
        gm[b] = g[b]
        one = run_gpu(n, layers, x, theta, gm, dtype=dtype, psi=False)
        check(dtype, f"dtheta[{b}]", one["dth"], G["dth"][k])


def test_ibm20_sampled():
    _sampled("ibm20")


def test_ionq20_sampled():
    _sampled("ionq20")


def test_zz26_sampled_against_oracle():
    _sampled("zz26")


def _closed_form(x, th):
    c = np.cos(x) * np.cos(th)
    n = len(c)
    out = np.empty(n)
    out[0] = np.prod(c[1:])
    for q in range(1, n):
        out[q] = np.prod(c[: q + 1])
    return out


def _check_closed_form(got, x, theta, g, n_theta):
    """<Z>, dx and d theta of a circuit whose <Z_q> is the prefix-parity
    product of c_j = cos x_j cos th_j (th = the first n entries of theta)."""
    B, n = g.shape
    dth_ref = np.zeros(n_theta)
    for b in range(B):
        c = np.cos(x[b]) * np.cos(theta[:n])
        ez = _closed_form(x[b], theta[:n])
        assert np.max(np.abs(got["ez"][b] - ez)) < ABS_C64
        dL_dc = np.zeros(n)
        for q in range(n):
            idx = list(range(1, n)) if q == 0 else list(range(q + 1))
            for j in idx:
                dL_dc[j] += g[b, q] * np.prod([c[i] for i in idx if i != j])
        dx = dL_dc * (-np.sin(x[b]) * np.cos(theta[:n]))
        assert np.max(np.abs(got["dx"][b] - dx)) < ABS_C64
        dth_ref[:n] += dL_dc * (-np.cos(x[b]) * np.sin(theta[:n]))
    assert np.max(np.abs(got["dth"] - dth_ref)) < ABS_C64 * B


def test_zz26_one_block_closed_form_full_size():
    """RX(x), RY(th), IsingZZ ring, CNOT ring at n = 26, B = 8: <Z_q> is a
    product of cos x_j cos th_j (the ring maps bits to prefix parities), and
    so are its derivatives; the ZZ angles do not enter."""
    n, B = 26, 8
    layers = W.zz_circuit(n, 1)
    x, theta, _ = W.draw_inputs(n, layers, B, seed=0)
    g = W.draw_upstream(B, n, seed=3)
    got = run_gpu(n, layers, x, theta, g, psi=False)
    _check_closed_form(got, x, theta, g, 2 * n)


def test_max_qubits_closed_form():
    """n = 30, the largest register the library accepts (2^30 amplitudes, 8 GiB
    per sample in complex64): [CNOT ring, RX(x), RY(th), CNOT ring] on |0..0>.
    The first ring leaves |0..0> as it is, so <Z> has the same closed form as
    one zz block; with no leading single-qubit layer every layer runs as its own
    pass (forward tile passes with the ring gathered into the first, the ring
    kernel, the backward ring with lambda formed in it, backward tile passes with
    the RX gradients folded into RY's).  Small angles keep the 30-factor products
    of order one."""
    n, B = 30, 1
    layers = [("CNOT_RING", "none", 0, 0), ("RX", "input", 0, 0), ("RY", "theta", 0, 0),
              ("CNOT_RING", "none", 0, 0)]
    rng = np.random.default_rng(30)
    x = rng.uniform(0.0, 0.4, size=(B, n))
    theta = rng.uniform(-0.4, 0.4, size=n)
    g = W.draw_upstream(B, n, seed=30)
    got = run_gpu(n, layers, x, theta, g, psi=False)
    assert np.allclose(got["norms"], 1.0, atol=1e-4)
    assert np.min(np.abs(got["ez"])) > 0.05
    _check_closed_form(got, x, theta, g, n)


def test_zz26_full_circuit_properties():
    cfg = W.WORKLOADS["zz26"]
    n, layers, B = cfg["n"], cfg["layers"](), cfg["batch"]
    x, theta, g = W.draw_inputs(n, layers, B, seed=0)
    a = run_gpu(n, layers, x, theta, g, psi=False)
    assert np.allclose(a["norms"], 1.0, atol=1e-5)
    assert np.all(np.abs(a["ez"]) <= 1.0 + 1e-6)
    del a
    b1 = run_gpu(n, layers, x, theta, g, psi=False)
    b2 = run_gpu(n, layers, x, theta, g, psi=False)
    assert np.array_equal(b1["dth"], b2["dth"]) and np.array_equal(b1["dx"], b2["dx"])
    # checkpoints off: same gradients within the c64 tolerance
    c0 = run_gpu(n, layers, x, theta, g, psi=False, ckpt=0)
    assert np.max(np.abs(c0["dx"] - b1["dx"])) < ABS_C64
    assert np.max(np.abs(c0["dth"] - b1["dth"])) < ABS_C64 * B

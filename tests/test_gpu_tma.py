"""TMA-staged tile passes (complex64) against the oracle and against the
per-thread-copy passes, through the C ABI.

The circuits are chosen so that the plan runs TMA passes of every form the
kernel has: contiguous first passes with 3 rounds (16-byte accesses in round
0), strided passes (c = 10, 9, 5), the backward diagonal undo in round 0
(identity and ring z maps), the forward diagonal phase in the last round, the
backward scatter through the CNOT ring, complex, real and brick gates."""
import re

import numpy as np
import pytest

from oracle import qsim_oracle as O
from paper_2506_04891_gb300 import workloads as W
from tests.gpu_helpers import ABS_C64, check, rel, run_gpu

pytestmark = pytest.mark.gpu

FAMILIES = {
    "zz": lambda n: W.zz_circuit(n, 2),
    "hea": lambda n: W.hea_circuit(n, 2),
    "ibm": lambda n: W.ibm_circuit(n, 2),
    "ionq": lambda n: W.ionq_circuit(n, 2),
    "qdi": lambda n: W.qdi_circuit(n, 2),
}


def _run(n, layers, x, theta, g, tma):
    import torch
    from paper_2506_04891_gb300 import qlayer as Q
    c = Q.Circuit(n, layers, dtype="c64", path=2, tuning={"tma": tma})
    plan = c.describe(g.shape[0])
    B = g.shape[0]
    xt = torch.tensor(x, device="cuda") if x.size else None
    tt = torch.tensor(theta, device="cuda") if theta.size else None
    psi, ez = c.forward(xt, tt, batch=B)
    dth, dx = c.backward(xt, tt, psi, torch.tensor(g, device="cuda"))
    torch.cuda.synchronize()
    out = dict(psi=psi.cpu().numpy().astype(np.complex128), ez=ez.cpu().numpy(), dth=dth.cpu().numpy(),
               dx=dx.cpu().numpy() if dx is not None else None, plan=plan)
    del c, psi
    torch.cuda.empty_cache()
    return out


@pytest.mark.parametrize("name", sorted(FAMILIES))
@pytest.mark.parametrize("n", [14, 15, 17])
def test_tma_passes_match_oracle_and_per_thread_copies(name, n):
    from paper_2506_04891_gb300 import qlayer as Q
    layers = FAMILIES[name](n)
    B = 2
    x, theta, g = W.draw_inputs(n, layers, B, seed=21)
    g = W.draw_upstream(B, n, seed=21)
    a = _run(n, layers, x, theta, g, 1)
    b = _run(n, layers, x, theta, g, 0)
    ntma = len(re.findall(r" tma=1", a["plan"]))
    assert ntma > 0, a["plan"]
    assert " tma=1" not in b["plan"]
    ez, dth, _, dx = O.adjoint(n, layers, x if x.size else np.zeros((B, 0)), theta, g)
    psi = O.forward(n, layers, x if x.size else np.zeros((B, 0)), theta)
    for got in (a, b):
        assert rel(got["psi"], psi) < 1e-5
        check("c64", "ez", got["ez"], ez)
        if dx.size:
            check("c64", "dx", got["dx"][:, : dx.shape[1]], dx)
        if dth.size:
            check("c64", "dtheta", got["dth"], dth, batch_sum=B)
    # the two copy paths agree well inside the complex64 tolerance (the TMA
    # passes run single-qubit gates in scaled form, the others in full form)
    assert np.max(np.abs(a["ez"] - b["ez"])) < 1e-5
    assert Q.qc_kernel_timeouts() == 0


def test_tma_plan_covers_the_zz26_backward_and_strided_forward():
    from paper_2506_04891_gb300 import qlayer as Q
    c = Q.Circuit(26, W.zz_circuit(26, 12), dtype="c64")
    plan = c.describe(8).splitlines()
    fwd = [l for l in plan if l.startswith("F ") and "TILE" in l]
    bwd = [l for l in plan if l.startswith("B ") and "TILE" in l]
    assert all(" tma=1" in l for l in bwd)
    assert sum(" tma=1" in l for l in fwd) == 22  # the ring-gathering passes keep per-thread copies


@pytest.mark.parametrize("case", ["near_cutoff", "exact_pi"])
def test_scaled_rotations_near_singular_angles(case):
    """Real (RY) passes run in scaled form (one packed FMA per output, the
    cosines carried as a factor); a pass falls back to the full form when a
    cosine is below 2^-10.  Angles with cos(theta/2) just above the cutoff
    (large tangents) and exactly at theta = pi (cosine ~ 6e-17: fallback)
    must both match the oracle."""
    n, B = 15, 2
    layers = W.zz_circuit(n, 3)
    x, theta, _ = W.draw_inputs(n, layers, B, seed=5)
    g = W.draw_upstream(B, n, seed=5)
    ry = [off for kind, src, off, _ in layers if kind == "RY"]
    if case == "near_cutoff":
        c = 1.5e-3  # tangent ~ 670
        for k, off in enumerate(ry):
            theta[off + 3 * k] = 2 * np.arccos(c)
            theta[off + 11] = 2 * np.arccos(-c)
    else:
        theta[ry[0] + 2] = np.pi
        theta[ry[1] + 14] = np.pi
    a = _run(n, layers, x, theta, g, 1)
    ez, dth, _, dx = O.adjoint(n, layers, x, theta, g)
    psi = O.forward(n, layers, x, theta)
    assert rel(a["psi"], psi) < 1e-5
    check("c64", "ez", a["ez"], ez)
    check("c64", "dx", a["dx"][:, : dx.shape[1]], dx)
    check("c64", "dtheta", a["dth"], dth, batch_sum=B)


@pytest.mark.parametrize("case", ["generic", "near_cutoff", "exact_pi"])
def test_scaled_complex_rotations(case):
    """Complex single-qubit passes with equal diagonal entries (RX, SX, GPI2)
    run in scaled form (one complex multiply-add per output, the diagonal
    carried as a factor, the last gate of a pass restoring it); a pass falls
    back to the full form when a diagonal entry is below 2^-10.  RX angles
    with cos(theta/2) just above the cutoff and exactly at theta = pi must
    match the oracle like generic ones."""
    n, B = 15, 2
    b = W._Builder(n)
    b.add("RX", "input")
    for _ in range(2):
        b.add("RX", "theta")
        b.add("CNOT_RING")
        b.add("GPI2", "theta")
        b.add("SX")
        b.add("CNOT_RING")
    layers = b.layers
    x, theta, _ = W.draw_inputs(n, layers, B, seed=6)
    g = W.draw_upstream(B, n, seed=6)
    rx = [off for kind, src, off, _ in layers if kind == "RX" and src == "theta"]
    if case == "near_cutoff":
        c = 1.5e-3
        for k, off in enumerate(rx):
            theta[off + 3 * k] = 2 * np.arccos(c)
            theta[off + 11] = 2 * np.arccos(-c)
    elif case == "exact_pi":
        theta[rx[0] + 2] = np.pi
        theta[rx[1] + 14] = np.pi
    a = _run(n, layers, x, theta, g, 1)
    assert len(re.findall(r" tma=1", a["plan"])) > 0, a["plan"]
    ez, dth, _, dx = O.adjoint(n, layers, x, theta, g)
    psi = O.forward(n, layers, x, theta)
    assert rel(a["psi"], psi) < 1e-5
    check("c64", "ez", a["ez"], ez)
    check("c64", "dx", a["dx"][:, : dx.shape[1]], dx)
    check("c64", "dtheta", a["dth"], dth, batch_sum=B)

"""The per-gate complex128 PyTorch comparison path (bench.py --impl pergate)
against the oracle on the CPU: same <Z>, d theta and d x to 1e-12 on every
circuit family, so the speedups stated against it compare equal work."""
import numpy as np
import pytest
import torch

import pergate_torch as PG
from oracle import qsim_oracle as O
from paper_2506_04891_gb300 import workloads as W

FAMILIES = {
    "hea": lambda n: W.hea_circuit(n, 2),
    "zz": lambda n: W.zz_circuit(n, 2),
    "ibm": lambda n: W.ibm_circuit(n, 2),
    "ionq": lambda n: W.ionq_circuit(n, 2),
    "qdi": lambda n: W.qdi_circuit(n, 2),
}


@pytest.mark.parametrize("name", sorted(FAMILIES))
@pytest.mark.parametrize("n", [2, 5])
def test_pergate_matches_oracle(name, n):
    layers = FAMILIES[name](n)
    B = 3
    x, theta, _ = W.draw_inputs(n, layers, B, seed=4)
    g = W.draw_upstream(B, n, seed=4)
    xt = torch.tensor(x) if x.size else None
    ez, dth, dx = PG.fwd_bwd(n, layers, xt, torch.tensor(theta), torch.tensor(g))
    ez_r, dth_r, _, dx_r = O.adjoint(n, layers, x if x.size else np.zeros((B, 0)), theta, g)
    assert np.max(np.abs(ez.numpy() - ez_r)) < 1e-12
    if theta.size:
        assert np.max(np.abs(dth.numpy() - dth_r)) < 1e-12
    if x.size:
        assert np.max(np.abs(dx.numpy() - dx_r)) < 1e-12


def test_max_batch_counts_every_gate():
    layers = W.zz_circuit(20, 12)
    assert PG.gate_count(20, layers) == 20 + 12 * 3 * 20
    assert PG.max_batch(20, layers, 200 * 2 ** 30, 8) == 8
    assert PG.max_batch(26, W.zz_circuit(26, 12), 200 * 2 ** 30, 8) == 0

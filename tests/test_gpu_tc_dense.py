"""Tensor-core dense block (qc_options.tc_dense, an experiment): the forward
pass of a real single-qubit layer on the 7 high bits of a tile as one
128 x 128 tcgen05 kind::tf32 matrix product with the 3xTF32 split, against the
oracle (complex64 tolerance) and against the register rounds."""
import numpy as np
import pytest

from oracle import qsim_oracle as O
from paper_2506_04891_gb300 import workloads as W
from tests.gpu_helpers import check, rel

pytestmark = pytest.mark.gpu

# n = 19: each RY layer runs a contiguous 12-bit pass and a strided pass on
# bits 12..18 (32 contiguous amplitudes, 7 gate bits): the tensor-core block
LAYERS19 = [("RX", "input", 0, 0), ("ECR_BRICK", "none", 0, 0), ("RY", "theta", 0, 0),
            ("ECR_BRICK", "none", 0, 1), ("RY", "theta", 19, 0)]


def _run(n, layers, x, theta, g, tc):
    import torch
    from paper_2506_04891_gb300 import qlayer as Q
    c = Q.Circuit(n, layers, dtype="c64", path=2, tuning={"tc_dense": tc})
    plan = c.describe(g.shape[0])
    xt, tt = torch.tensor(x, device="cuda"), torch.tensor(theta, device="cuda")
    psi, ez = c.forward(xt, tt, batch=g.shape[0])
    dth, dx = c.backward(xt, tt, psi, torch.tensor(g, device="cuda"))
    torch.cuda.synchronize()
    out = dict(psi=psi.cpu().numpy().astype(np.complex128), ez=ez.cpu().numpy(), dth=dth.cpu().numpy(),
               dx=dx.cpu().numpy(), plan=plan, timeouts=Q.qc_kernel_timeouts())
    del c, psi
    torch.cuda.empty_cache()
    return out


def test_tc_dense_block_matches_oracle_and_register_rounds():
    n, B = 19, 2
    x, theta, _ = W.draw_inputs(n, LAYERS19, B, seed=9)
    g = W.draw_upstream(B, n, seed=9)
    a = _run(n, LAYERS19, x, theta, g, 1)
    b = _run(n, LAYERS19, x, theta, g, 0)
    assert a["plan"].count(" tc=1") == 2 and " tc=1" not in b["plan"]
    assert a["timeouts"] == 0
    ez, dth, _, dx = O.adjoint(n, LAYERS19, x, theta, g)
    psi = O.forward(n, LAYERS19, x, theta)
    for got in (a, b):
        assert rel(got["psi"], psi) < 1e-5
        check("c64", "ez", got["ez"], ez)
        check("c64", "dx", got["dx"], dx)
        check("c64", "dtheta", got["dth"], dth, batch_sum=B)
    assert np.max(np.abs(a["psi"] - b["psi"])) < 2e-6


def test_tc_dense_block_on_the_zz26_golden_sample():
    """zz26's 11 strided forward passes on the tensor cores, sample 0 against
    the oracle's stored values."""
    import os
    G = np.load(os.path.join(os.path.dirname(__file__), "golden", "zz26.npz"))
    cfg = W.WORKLOADS["zz26"]
    n, layers = cfg["n"], cfg["layers"]()
    x, theta, g = W.draw_inputs(n, layers, cfg["batch"], seed=0)
    bs = [int(v) for v in G["samples"]]
    a = _run(n, layers, x[bs], theta, g[bs], 1)
    assert a["plan"].count(" tc=1") == 11 and a["timeouts"] == 0
    assert np.max(np.abs(a["ez"] - G["ez"])) <= 2e-5
    assert np.max(np.abs(a["dx"] - G["dx"])) <= 2e-5
    assert np.max(np.abs(a["dth"] - G["dth"].sum(axis=0))) <= 2e-5 * len(bs)
    got = np.stack([a["psi"][k][G["psi_idx"][k]] for k in range(len(bs))])
    assert np.max(np.abs(got - G["psi_val"])) <= 2e-5

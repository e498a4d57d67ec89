"""After qc_create, the compute calls allocate nothing and never synchronise
the device: the plan tables travel into the caller's workspace with every
call, and qc_expect_z reuses the scratch qc_create allocated (in sample chunks
when the batch is larger than it holds)."""
import numpy as np
import pytest

from oracle import qsim_oracle as O
from paper_2506_04891_gb300 import workloads as W
from tests.gpu_helpers import ABS_C64

pytestmark = pytest.mark.gpu


def test_forward_backward_expect_make_no_allocation_at_new_batch_sizes():
    import torch
    from paper_2506_04891_gb300 import qlayer as Q
    n = 14
    layers = W.hea_circuit(n, 2)
    c = Q.Circuit(n, layers, dtype="c64", path=2)
    a0 = Q.qc_alloc_count()
    for B in (1, 3, 5, 2, 3):
        x, th, g = W.draw_inputs(n, layers, B, seed=B)
        xt, tt = torch.tensor(x, device="cuda"), torch.tensor(th, device="cuda")
        ws = torch.empty(c.workspace_bytes(B), dtype=torch.uint8, device="cuda")
        psi, ez = c.forward(xt, tt, workspace=ws)
        ez2 = c.expect_z(psi)
        dth, dx = c.backward(xt, tt, psi, torch.tensor(g, device="cuda"), workspace=ws)
        torch.cuda.synchronize()
        ref_ez, ref_dth, _, ref_dx = O.adjoint(n, layers, x, th, g)
        assert np.max(np.abs(ez.cpu().numpy() - ref_ez)) <= ABS_C64
        assert np.max(np.abs(ez2.cpu().numpy() - ref_ez)) <= ABS_C64
        assert np.max(np.abs(dx.cpu().numpy() - ref_dx)) <= ABS_C64
        assert np.max(np.abs(dth.cpu().numpy() - ref_dth)) <= ABS_C64 * B
    assert Q.qc_alloc_count() == a0


def test_expect_z_chunks_large_batches_through_its_fixed_scratch():
    """n = 24: one sample fills 2^10 CTAs x 25 partial sums (200 KB), so the
    2 MiB scratch holds 10 samples and a batch of 23 runs in three launches."""
    import torch
    from paper_2506_04891_gb300 import qlayer as Q
    n, B = 24, 23
    c = Q.Circuit(n, [("RX", "input", 0, 0)], dtype="c64")
    x = np.random.default_rng(3).uniform(0, np.pi, size=(B, n))
    psi, ez = c.forward(torch.tensor(x, device="cuda"), None, batch=B)
    a0 = Q.qc_alloc_count()
    ez2 = c.expect_z(psi)
    torch.cuda.synchronize()
    assert Q.qc_alloc_count() == a0
    # product state: <Z_q> = cos x_q (closed form)
    assert np.max(np.abs(ez2.cpu().numpy() - np.cos(x))) <= ABS_C64
    assert np.array_equal(ez2.cpu().numpy(), ez.cpu().numpy())

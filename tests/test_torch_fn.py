"""torch.autograd integration: gradients of a loss through QuantumLayer match
the oracle's adjoint; an optimiser step runs."""
import numpy as np
import pytest

from paper_2506_04891_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,n", [("c128", 10), ("c64", 15)])
def test_autograd_matches_oracle(dtype, n):
    import torch
    from oracle import qsim_oracle as O
    from paper_2506_04891_gb300.torch_fn import QuantumLayer
    layers = W.zz_circuit(n, 2)
    x_np, theta_np, _ = W.draw_inputs(n, layers, 3, seed=21)
    layer = QuantumLayer(n, layers, dtype=dtype, theta=theta_np)
    x = torch.tensor(x_np, device="cuda", requires_grad=True)
    ez = layer(x)
    w = torch.linspace(-1, 1, n, dtype=torch.float64, device="cuda")
    loss = (ez * w).sum()
    loss.backward()
    g = np.tile(w.cpu().numpy(), (3, 1))
    ez_ref, dth_ref, _, dx_ref = O.adjoint(n, layers, x_np, theta_np, g)
    tol = 1e-11 if dtype == "c128" else 2e-5
    assert np.max(np.abs(ez.detach().cpu().numpy() - ez_ref)) < tol
    assert np.max(np.abs(x.grad.cpu().numpy() - dx_ref)) < tol
    assert np.max(np.abs(layer.theta.grad.cpu().numpy() - dth_ref)) < tol * 3


def test_training_step_and_checkpoint_guard():
    import torch
    from paper_2506_04891_gb300.torch_fn import QuantumLayer
    n = 22  # 2 x 2^22 x 8 B states: checkpoints stay off (below 1 GiB)
    layers = W.zz_circuit(n, 2)
    layer = QuantumLayer(n, layers, dtype="c64", seed=3)
    opt = torch.optim.SGD(layer.parameters(), lr=0.1)
    x = torch.rand((2, n), dtype=torch.float64, device="cuda")
    before = layer.theta.detach().clone()
    loss = layer(x).mean()
    loss.backward()
    opt.step()
    assert not torch.equal(before, layer.theta.detach())
    # with checkpoints, a second forward before the first backward is refused
    ck = QuantumLayer(14, W.zz_circuit(14, 3), dtype="c64", ckpt_every=2, seed=4, path=2)
    assert ck.circuit.uses_checkpoints(2)
    xa = torch.rand((2, 14), dtype=torch.float64, device="cuda")
    la = ck(xa).sum()
    lb = ck(xa * 0.5).sum()
    with pytest.raises(RuntimeError):
        la.backward()
    lb.backward()

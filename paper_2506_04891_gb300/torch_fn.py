"""torch.autograd integration of the C ABI.

``QLayerFunction`` maps (x, theta) to <Z> (batch x n) with qc_forward and
returns gradients with qc_backward (the adjoint sweep).  ``QuantumLayer`` is a
torch.nn.Module holding theta as a parameter.  Every computation runs in the
CUDA library; this module only moves tensors and keeps the forward's state for
the backward.
"""
from __future__ import annotations

import torch

from . import qlayer as Q


class QLayerFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, circuit: "Q.Circuit", x: torch.Tensor, theta: torch.Tensor):
        batch = x.shape[0]
        psi, ez = circuit.forward(x, theta, batch=batch)
        circuit._fwd_gen = getattr(circuit, "_fwd_gen", 0) + 1
        ctx.circuit = circuit
        ctx.gen = circuit._fwd_gen
        ctx.x_dtype = x.dtype
        ctx.t_dtype = theta.dtype
        ctx.save_for_backward(x, theta, psi)
        return ez.to(device=x.device, dtype=x.dtype)

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        x, theta, psi = ctx.saved_tensors
        circ = ctx.circuit
        if circ.uses_checkpoints(x.shape[0]) and circ._fwd_gen != ctx.gen:
            raise RuntimeError("another forward of this circuit ran since this output was computed; "
                               "with re-anchoring checkpoints the backward must follow its forward "
                               "(or create the circuit with ckpt_every=0)")
        dth, dx = circ.backward(x, theta, psi, g.contiguous())
        gx = dx.to(device=x.device, dtype=ctx.x_dtype) if ctx.needs_input_grad[1] and dx is not None else None
        gt = dth.to(device=theta.device, dtype=ctx.t_dtype) if ctx.needs_input_grad[2] else None
        return None, gx, gt


class QuantumLayer(torch.nn.Module):
    """<Z_q> of a layered circuit as a differentiable layer: forward(x) -> [B, n]."""

    def __init__(self, n: int, layers, dtype: str = "c64", theta=None, ckpt_every: int = -1,
                 seed: int = 0, device: str = "cuda", path: int = 0):
        super().__init__()
        self.circuit = Q.Circuit(n, layers, dtype=dtype, ckpt_every=ckpt_every, path=path)
        if theta is None:
            gen = torch.Generator().manual_seed(seed)
            theta = 2 * torch.pi * torch.rand(self.circuit.n_theta, generator=gen, dtype=torch.float64)
        self.theta = torch.nn.Parameter(torch.as_tensor(theta, dtype=torch.float64).clone().to(device))

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        return QLayerFunction.apply(self.circuit, x, self.theta)

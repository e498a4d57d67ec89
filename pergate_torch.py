"""Plain complex128 per-gate PyTorch path on the GPU: the speedup denominator.

This is the way a PyTorch state-vector simulator applies a circuit when it
does not specialise anything: every gate of every layer is applied on its own
by ``torch.einsum`` over that gate's qubit axes of the batch state reshaped to
``[B, 2, ..., 2]`` (the Sequential Einsum technique of Sec. 2.2.2, run on the
GPU), in complex128, and the gradient of the measured <Z> comes from
``torch.autograd`` (backpropagation through every gate application, the
paper's own differentiation route; Sec. 3).  Gate matrices follow Appendix A
with the same two readings the library uses (MS entry (3,0) with the
conjugate phase; ECR = (I(x)X - X(x)Y)/sqrt(2)).

It is a comparison program for ``bench.py --impl pergate``: the library never
imports it, and it shares no code with the CUDA path or with the oracle (a CPU
test checks it against the oracle on small circuits).  Autograd keeps the
input of every gate application, so its memory is about (gates + 2) x the
batch state; ``max_batch`` gives the largest batch that fits a byte budget.
"""
from __future__ import annotations

import math
import string

import torch

LETTERS = string.ascii_letters  # einsum subscripts: batch + up to 51 qubit axes


def _cplx(re, im=None):
    if im is None:
        im = torch.zeros_like(re)
    return torch.complex(re, im)


def _phase(a):
    """exp(i a) for a real tensor a."""
    return torch.complex(torch.cos(a), torch.sin(a))


def gate_1q(kind: str, t):
    """2x2 (or [B, 2, 2]) matrix of a single-qubit gate with parameter tensor t."""
    one = torch.ones_like(t)
    zero = torch.zeros_like(t)
    if kind == "RX":
        c, s = _cplx(torch.cos(t / 2)), _cplx(zero, -torch.sin(t / 2))
        rows = [[c, s], [s, c]]
    elif kind == "RY":
        c, s = _cplx(torch.cos(t / 2)), _cplx(torch.sin(t / 2))
        rows = [[c, -s], [s, c]]
    elif kind == "RZ":
        rows = [[_phase(-t / 2), _cplx(zero)], [_cplx(zero), _phase(t / 2)]]
    elif kind == "GPI":
        rows = [[_cplx(zero), _phase(-2 * math.pi * t)], [_phase(2 * math.pi * t), _cplx(zero)]]
    elif kind == "GPI2":
        r = 1 / math.sqrt(2.0)
        mi = _cplx(zero, -one)
        rows = [[_cplx(one * r), mi * _phase(-2 * math.pi * t) * r],
                [mi * _phase(2 * math.pi * t) * r, _cplx(one * r)]]
    else:
        raise ValueError(kind)
    return torch.stack([torch.stack(r, dim=-1) for r in rows], dim=-2)


def gate_const(kind: str, device):
    c = torch.complex128
    r2 = 1 / math.sqrt(2.0)
    if kind == "X":
        m = [[0, 1], [1, 0]]
    elif kind == "SX":
        m = [[0.5 + 0.5j, 0.5 - 0.5j], [0.5 - 0.5j, 0.5 + 0.5j]]
    elif kind == "Z":
        m = [[1, 0], [0, -1]]
    elif kind == "S":
        m = [[1, 0], [0, 1j]]
    elif kind == "H":
        m = [[r2, r2], [r2, -r2]]
    elif kind == "CNOT":
        m = [[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]]
    elif kind == "CZ":
        m = [[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, -1]]
    elif kind == "SWAP":
        m = [[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]]
    elif kind == "ECR":
        # (I (x) X - X (x) Y) / sqrt(2), first qubit the left factor
        m = [[0, r2, 0, 1j * r2], [r2, 0, -1j * r2, 0], [0, 1j * r2, 0, r2], [-1j * r2, 0, r2, 0]]
    else:
        raise ValueError(kind)
    return torch.tensor(m, dtype=c, device=device)


def gate_isingzz(t):
    a, b = _phase(-t / 2), _phase(t / 2)
    z = _cplx(torch.zeros_like(t))
    d = [a, b, b, a]
    return torch.stack([torch.stack([d[i] if i == j else z for j in range(4)], dim=-1) for i in range(4)], dim=-2)


def gate_ms(p0, p1, th):
    c = _cplx(torch.cos(math.pi * th))
    s = torch.sin(math.pi * th)
    z = _cplx(torch.zeros_like(th))
    mi_s = _cplx(torch.zeros_like(th), -s)
    e03 = mi_s * _phase(-2 * math.pi * (p0 + p1))
    e12 = mi_s * _phase(-2 * math.pi * (p1 - p0))
    e21 = mi_s * _phase(-2 * math.pi * (p0 - p1))
    e30 = mi_s * _phase(2 * math.pi * (p0 + p1))
    rows = [[c, z, z, e03], [z, c, e12, z], [z, e21, c, z], [e30, z, z, c]]
    return torch.stack([torch.stack(r, dim=-1) for r in rows], dim=-2)


def _brick_pairs(n, parity):
    return [(parity + 2 * i, parity + 2 * i + 1) for i in range(max(0, (n - parity) // 2))]


def _apply(psi, M, qubits, n, per_sample):
    """One gate by einsum over its qubit axes (axis 1 + q holds qubit q)."""
    st = LETTERS[: n + 1]  # st[0] = batch
    k = len(qubits)
    outs = LETTERS[n + 1: n + 1 + k]
    ins = "".join(st[1 + q] for q in qubits)
    res = list(st)
    for j, q in enumerate(qubits):
        res[1 + q] = outs[j]
    if k == 2:
        M = M.reshape(M.shape[:-2] + (2, 2, 2, 2))
    gs = (st[0] if per_sample else "") + outs + ins
    return torch.einsum(f"{gs},{st}->{''.join(res)}", M, psi)


def _params(source, offset, count, x, theta):
    if source == "theta":
        return theta[offset: offset + count], False
    if source == "input":
        return x[:, offset: offset + count], True
    return None, False


def forward(n, layers, x, theta, batch):
    """psi [B, 2, ..., 2] complex128 after every gate, and <Z> [B, n]."""
    dev = theta.device if theta is not None else (x.device if x is not None else "cuda")
    psi = torch.zeros((batch,) + (2,) * n, dtype=torch.complex128, device=dev)
    psi[(slice(None),) + (0,) * n] = 1.0
    for kind, source, offset, parity in layers:
        if kind in ("RX", "RY", "RZ", "GPI", "GPI2"):
            p, ps = _params(source, offset, n, x, theta)
            for q in range(n):
                t = (p[:, q] if ps else p[q]) if p is not None else torch.zeros((), dtype=torch.float64, device=dev)
                psi = _apply(psi, gate_1q(kind, t), (q,), n, ps)
        elif kind == "ISINGZZ_RING":
            p, ps = _params(source, offset, n, x, theta)
            for j in range(n):
                t = (p[:, j] if ps else p[j]) if p is not None else torch.zeros((), dtype=torch.float64, device=dev)
                psi = _apply(psi, gate_isingzz(t), (j, (j + 1) % n), n, ps)
        elif kind == "CNOT_RING":
            U = gate_const("CNOT", dev)
            for q in range(n):
                psi = _apply(psi, U, (q, (q + 1) % n), n, False)
        elif kind in ("X", "SX", "Z", "S", "H"):
            U = gate_const(kind, dev)
            for q in range(n):
                psi = _apply(psi, U, (q,), n, False)
        elif kind in ("ECR_BRICK", "CZ_BRICK", "SWAP_BRICK"):
            U = gate_const(kind.split("_")[0], dev)
            for pair in _brick_pairs(n, parity):
                psi = _apply(psi, U, pair, n, False)
        elif kind == "MS_BRICK":
            pairs = _brick_pairs(n, parity)
            p, ps = _params(source, offset, 3 * len(pairs), x, theta)
            for i, pair in enumerate(pairs):
                if p is None:
                    z = torch.zeros((), dtype=torch.float64, device=dev)
                    a, b, c = z, z, z
                elif ps:
                    a, b, c = p[:, 3 * i], p[:, 3 * i + 1], p[:, 3 * i + 2]
                else:
                    a, b, c = p[3 * i], p[3 * i + 1], p[3 * i + 2]
                psi = _apply(psi, gate_ms(a, b, c), pair, n, ps)
        else:
            raise ValueError(f"layer kind {kind!r} is not in the per-gate path")
    prob = (psi.real ** 2 + psi.imag ** 2)
    ez = []
    for q in range(n):
        m = prob.movedim(1 + q, 1).reshape(batch, 2, -1).sum(dim=2)
        ez.append(m[:, 0] - m[:, 1])
    return psi, torch.stack(ez, dim=1)


def fwd_bwd(n, layers, x, theta, g):
    """One evaluation: forward, <Z>, and d/d(theta, x) of sum(g * <Z>) by
    autograd.  Returns (ez, d_theta, d_x) as detached tensors."""
    xx = x.detach().clone().requires_grad_(x.numel() > 0) if x is not None else None
    tt = theta.detach().clone().requires_grad_(theta.numel() > 0) if theta is not None else None
    B = g.shape[0]
    _, ez = forward(n, layers, xx, tt, B)
    loss = (ez * g).sum()
    leaves = [v for v in (tt, xx) if v is not None and v.requires_grad]
    grads = torch.autograd.grad(loss, leaves) if leaves else []
    gi = iter(grads)
    dth = next(gi) if tt is not None and tt.requires_grad else None
    dx = next(gi) if xx is not None and xx.requires_grad else None
    return ez.detach(), dth, dx


def gate_count(n, layers):
    c = 0
    for kind, _s, _o, parity in layers:
        c += len(_brick_pairs(n, parity)) if kind.endswith("_BRICK") else n
    return c


def max_batch(n, layers, budget_bytes, want):
    """Largest batch <= want whose autograd footprint (every gate's input kept,
    plus a few working states) fits budget_bytes."""
    per = (gate_count(n, layers) + 4) * (16 << n)
    return max(0, min(want, int(budget_bytes // per)))

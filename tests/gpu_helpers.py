"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and compare against the oracle with the stated tolerances."""
import numpy as np

# Tolerances (stated for the method):
#   complex128: relative 1e-12 per output tensor, ||gpu - ref|| / ||ref||
#   complex64:  absolute 2e-5 on <Z> and on per-sample gradients with the
#               upstream gradient g = 1/n; batch-summed d theta: 2e-5 * B
REL_C128 = 1e-12
ABS_C64 = 2e-5


def run_gpu(n, layers, x, theta, g, dtype="c64", path=0, fuse=1, ckpt=-1, psi=True, psi_idx=None):
    """Forward (+ <Z>) and adjoint backward on the GPU.

    psi=True copies the whole state to the host; psi_idx={b: indices} returns
    only those amplitudes.  Norms of every sample are always returned."""
    import torch
    from paper_2506_04891_gb300 import qlayer as Q
    circ = Q.Circuit(n, layers, dtype=dtype, ckpt_every=ckpt, path=path, fuse=fuse)
    B = g.shape[0]
    xt = torch.tensor(x, dtype=torch.float64, device="cuda") if x is not None and x.size else None
    tt = torch.tensor(theta, dtype=torch.float64, device="cuda") if theta is not None and theta.size else None
    gt = torch.tensor(g, dtype=torch.float64, device="cuda")
    ps, ez = circ.forward(xt, tt, batch=B)
    dth, dx = circ.backward(xt, tt, ps, gt)
    torch.cuda.synchronize()
    out = dict(ez=ez.cpu().numpy(), dth=dth.cpu().numpy(), dx=dx.cpu().numpy() if dx is not None else None)
    out["norms"] = (ps.abs().double() ** 2).sum(dim=1).cpu().numpy()
    if psi:
        out["psi"] = ps.cpu().numpy().astype(np.complex128)
    if psi_idx:
        out["psi_sel"] = {b: ps[b][torch.as_tensor(np.asarray(i), device="cuda")].cpu().numpy().astype(np.complex128)
                          for b, i in psi_idx.items()}
    del ps, ez, dth, dx, circ
    torch.cuda.empty_cache()
    return out


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    d = np.linalg.norm((a - b).ravel())
    r = np.linalg.norm(b.ravel())
    return d / r if r > 0 else d


def check(dtype, name, got, ref, batch_sum=1):
    got = np.asarray(got)
    ref = np.asarray(ref)
    assert got.shape == ref.shape, (name, got.shape, ref.shape)
    if ref.size == 0:
        return
    if dtype == "c128":
        r = rel(got, ref)
        assert r <= REL_C128, f"{name}: relative error {r:.3e} > {REL_C128}"
    else:
        e = np.max(np.abs(got - ref))
        tol = ABS_C64 * batch_sum
        assert e <= tol, f"{name}: max abs error {e:.3e} > {tol:.1e}"

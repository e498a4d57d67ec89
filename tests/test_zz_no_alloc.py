"""qc_expect_z_noalloc: the <Z> entry point for callers that cannot allocate.

Some callers cannot call cudaMalloc where they measure <Z>, because another
allocator holds their device memory or because an allocation's possible
device-wide synchronisation is not acceptable in their loop.  This entry point
keeps its partial sums in a fixed array inside the library's device image.  The
test calls it through the C ABI, twice in a row per case, and checks the result
against qc_expect_z within the tolerances used by the other GPU tests. It also
checks that a request beyond the array's limit is refused with a clear error.
The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2506_04891_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ABS_C64 = 2e-5
REL_C128 = 1e-12


def _noalloc_fn(Q):
    lib = ctypes.CDLL(Q.LIB_PATH)
    fn = lib.qc_expect_z_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return fn


@pytest.mark.parametrize("n,batch,dtype,depth", [(26, 8, "c64", 1), (14, 64, "c128", 2), (5, 3, "c64", 2)])
def test_expect_z_noalloc_matches_expect_z(n, batch, dtype, depth):
    import torch
    from paper_2506_04891_gb300 import qlayer as Q
    fn = _noalloc_fn(Q)
    layers = W.zz_circuit(n, depth)
    x, theta, _ = W.draw_inputs(n, layers, batch, seed=11)
    circ = Q.Circuit(n, layers, dtype=dtype)
    psi, _ = circ.forward(torch.tensor(x, device="cuda"), torch.tensor(theta, device="cuda"), ez=False)
    ref = circ.expect_z(psi)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        ez = torch.full((batch, n), float("nan"), dtype=torch.float64, device="cuda")
        st = fn(circ.handle, batch, psi.data_ptr(), ez.data_ptr(), stream)
        assert st == 0, Q.qc_last_error()
        torch.cuda.synchronize()
        got = ez.cpu().numpy()
        if dtype == "c128":
            r = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert r <= REL_C128, (call, r)
        else:
            assert np.max(np.abs(got - ref)) <= ABS_C64, call
    del psi, circ
    torch.cuda.empty_cache()


def test_expect_z_noalloc_rejects_oversized_requests():
    import torch
    from paper_2506_04891_gb300 import qlayer as Q
    fn = _noalloc_fn(Q)
    n, batch = 26, 16  # 16 * 2^12 * 27 partial sums > 2^20
    circ = Q.Circuit(n, [("RX", "input", 0, 0)], dtype="c64")
    dummy = torch.empty(2, dtype=torch.complex64, device="cuda")
    ez = torch.empty((batch, n), dtype=torch.float64, device="cuda")
    st = fn(circ.handle, batch, dummy.data_ptr(), ez.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 1
    assert "static scratch" in Q.qc_last_error()

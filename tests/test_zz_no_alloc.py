"""qc_expect_z_noalloc: the <Z> entry point for callers that cannot allocate.

Some callers cannot have device memory allocated where they measure <Z>:
another allocator (a framework's caching pool, a budget fixed at start-up)
holds their device memory, or a cudaMalloc's possible device-wide
synchronisation is not acceptable inside their loop.  This entry point keeps
its partial sums in a fixed array inside the library's device image.  The
tests call it through the C ABI, twice in a row per case, and check the result
against qc_expect_z within the tolerances of the other GPU tests; they check
that the calls leave the device's free memory unchanged, also in a fresh
process with lazy module loading (where a module is otherwise loaded, and its
arrays allocated, at first use), and that a request beyond the array's limit
is refused with a clear error.  The file is named so that pytest collects it
last.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2506_04891_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ABS_C64 = 2e-5
REL_C128 = 1e-12
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("n,batch,dtype,depth", [(26, 8, "c64", 1), (14, 64, "c128", 2), (5, 3, "c64", 2)])
def test_expect_z_noalloc_matches_expect_z(n, batch, dtype, depth):
    import torch
    from paper_2506_04891_gb300 import qlayer as Q
    layers = W.zz_circuit(n, depth)
    x, theta, _ = W.draw_inputs(n, layers, batch, seed=11)
    circ = Q.Circuit(n, layers, dtype=dtype)
    psi, _ = circ.forward(torch.tensor(x, device="cuda"), torch.tensor(theta, device="cuda"), ez=False)
    ref = circ.expect_z(psi)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    stream = torch.cuda.current_stream().cuda_stream
    outs = [torch.full((batch, n), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for call in range(2):
        Q.qc_expect_z_noalloc(circ.handle, batch, psi.data_ptr(), outs[call].data_ptr(), stream)
        torch.cuda.synchronize()
        got = outs[call].cpu().numpy()
        if dtype == "c128":
            r = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert r <= REL_C128, (call, r)
        else:
            assert np.max(np.abs(got - ref)) <= ABS_C64, call
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_reserved() == reserved0
    del psi, circ
    torch.cuda.empty_cache()


def test_expect_z_noalloc_rejects_oversized_requests():
    import torch
    from paper_2506_04891_gb300 import qlayer as Q
    n, batch = 26, 16  # 16 * 2^12 * 27 partial sums > 2^20
    circ = Q.Circuit(n, [("RX", "input", 0, 0)], dtype="c64")
    dummy = torch.empty(2, dtype=torch.complex64, device="cuda")
    ez = torch.empty((batch, n), dtype=torch.float64, device="cuda")
    with pytest.raises(Q.QCError) as e:
        Q.qc_expect_z_noalloc(circ.handle, batch, dummy.data_ptr(), ez.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
    assert e.value.status == 1
    assert "static scratch" in str(e.value)


_FRESH = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2506_04891_gb300 import qlayer as Q
from paper_2506_04891_gb300 import workloads as W
n, B = 12, 5
torch.cuda.init()
torch.zeros(1, device="cuda")
c = Q.Circuit(n, [("RX", "input", 0, 0)], dtype="c64")
x = np.random.default_rng(7).uniform(0, np.pi, size=(B, n))
psi, _ = c.forward(torch.tensor(x, device="cuda"), None, batch=B, ez=False)
ez = [torch.empty((B, n), dtype=torch.float64, device="cuda") for _ in range(2)]
torch.cuda.synchronize()
free0, _ = torch.cuda.mem_get_info()
for k in range(2):
    Q.qc_expect_z_noalloc(c.handle, B, psi.data_ptr(), ez[k].data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
free1, _ = torch.cuda.mem_get_info()
err = max(float(np.max(np.abs(e.cpu().numpy() - np.cos(x)))) for e in ez)
print("free", free0, free1, "err", err)
assert free1 == free0, (free0, free1)
assert err <= 2e-5, err
"""


def test_expect_z_noalloc_first_calls_allocate_nothing_with_lazy_loading():
    """A fresh process with CUDA_MODULE_LOADING=LAZY: qc_create did the set-up,
    so even the first two calls leave the free device memory unchanged."""
    env = dict(os.environ, CUDA_MODULE_LOADING="LAZY")
    r = subprocess.run([sys.executable, "-c", _FRESH, ROOT], capture_output=True, text=True, env=env,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]

"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Sizes are chosen so the oracle finishes in seconds while the layer path still
spans several tiles (n = 14, 15: two tile passes with a ragged second pass;
complex128 n = 13: tiles of 2^11), plus every edge the planner has: n = 1 and
2, empty circuits, batch 1, leading layers fused into the product state,
checkpoints, brick parities and the shared-memory whole-circuit path.
"""
import numpy as np
import pytest

from oracle import qsim_oracle as O
from paper_2506_04891_gb300 import workloads as W
from tests.gpu_helpers import ABS_C64, check, rel, run_gpu

pytestmark = pytest.mark.gpu


def oracle_all(n, layers, x, theta, g):
    B = g.shape[0]
    xx = x if x.size else np.zeros((B, 0))
    ez, dth, dth_s, dx = O.adjoint(n, layers, xx, theta, g)
    psi = O.forward(n, layers, xx, theta)
    return dict(ez=ez, dth=dth, dx=dx, psi=psi)


def compare(dtype, n, layers, B, seed=0, path=0, fuse=1, ckpt=-1, g=None):
    x, theta, g0 = W.draw_inputs(n, layers, B, seed=seed)
    g = g0 if g is None else g
    ref = oracle_all(n, layers, x, theta, g)
    got = run_gpu(n, layers, x, theta, g, dtype=dtype, path=path, fuse=fuse, ckpt=ckpt)
    if dtype == "c128":
        check(dtype, "psi", got["psi"], ref["psi"])
    else:
        r = rel(got["psi"], ref["psi"])
        assert r < 1e-5, f"psi relative error {r:.2e}"
    check(dtype, "ez", got["ez"], ref["ez"])
    check(dtype, "dx", got["dx"][:, : ref["dx"].shape[1]], ref["dx"])
    check(dtype, "dtheta", got["dth"], ref["dth"], batch_sum=B)
    return got, ref


CIRCUITS = {
    "hea": lambda n: W.hea_circuit(n, 2),
    "hea_ry": lambda n: W.hea_circuit(n, 2, block=("RY",)),
    "zz": lambda n: W.zz_circuit(n, 2),
    "ibm": lambda n: W.ibm_circuit(n, 2),
    "ionq": lambda n: W.ionq_circuit(n, 2),
}


def test_hea4_config_exact_c128():
    cfg = W.WORKLOADS["hea4"]
    for path in (0, 1, 2):
        compare("c128", 4, cfg["layers"](), cfg["batch"], path=path)


@pytest.mark.parametrize("name", sorted(CIRCUITS))
@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("path", [1, 2])
def test_small_circuits_both_paths(name, dtype, path):
    n = 7
    compare(dtype, n, CIRCUITS[name](n), 3, seed=1, path=path)


@pytest.mark.parametrize("name", sorted(CIRCUITS))
@pytest.mark.parametrize("dtype,n", [("c64", 14), ("c64", 15), ("c128", 13)])
def test_layer_path_multi_tile(name, dtype, n):
    compare(dtype, n, CIRCUITS[name](n), 2, seed=2, path=2)


@pytest.mark.parametrize("dtype,n", [("c64", 10), ("c64", 12), ("c128", 11), ("c64", 13)])
def test_diagonal_undone_in_the_backward_ring_pass(dtype, n):
    """HEA blocks: the first RZ of a block is undone and differentiated in the
    backward ring pass (whole-state rings at n = 10..12, tiled at 13)."""
    from paper_2506_04891_gb300 import qlayer as Q
    layers = W.hea_circuit(n, 3)
    d = Q.Circuit(n, layers, dtype=dtype, path=2).describe(3)
    assert any(l.startswith("B") and " RING " in l and "pre=1" in l for l in d.splitlines()), d
    compare(dtype, n, layers, 3, seed=16, path=2)


@pytest.mark.parametrize("name", sorted(CIRCUITS))
@pytest.mark.parametrize("n", [2, 3])
@pytest.mark.parametrize("path", [1, 2])
def test_every_circuit_family_at_n2_n3(name, n, path):
    compare("c128", n, CIRCUITS[name](n), 2, seed=12, path=path)


@pytest.mark.parametrize("fuse,ckpt", [(0, 0), (1, 0), (0, 2), (1, 3), (1, 1)])
@pytest.mark.parametrize("name", ["zz", "hea", "ibm"])
def test_layer_path_fusion_and_checkpoints(fuse, ckpt, name):
    n = 14
    layers = {"zz": W.zz_circuit(n, 3), "hea": W.hea_circuit(n, 3), "ibm": W.ibm_circuit(n, 3)}[name]
    compare("c64", n, layers, 2, seed=3, path=2, fuse=fuse, ckpt=ckpt)


@pytest.mark.parametrize("n", [1, 2, 3])
@pytest.mark.parametrize("path", [1, 2])
def test_tiny_n(n, path):
    layers = [("RX", "input", 0, 0), ("RY", "theta", 0, 0), ("GPI2", "theta", n, 0),
              ("RZ", "theta", 2 * n, 0), ("GPI", "theta", 3 * n, 0), ("SX", "none", 0, 0),
              ("X", "none", 0, 0)]
    if n >= 2:
        layers += [("ISINGZZ_RING", "theta", 4 * n, 0), ("CNOT_RING", "none", 0, 0),
                   ("MS_BRICK", "theta", 5 * n, 0), ("ECR_BRICK", "none", 0, 0),
                   ("RY", "theta", 8 * n, 0)]
    compare("c128", n, layers, 2, seed=4, path=path)


def test_every_kind_in_every_position_layer_path():
    n = 14
    kinds = ["RX", "RY", "RZ", "ISINGZZ_RING", "CNOT_RING", "X", "SX", "GPI", "GPI2",
             "MS_BRICK", "ECR_BRICK", "Z", "S", "H", "CZ_BRICK", "SWAP_BRICK", "ROT"]
    fixed = ("CNOT_RING", "X", "SX", "ECR_BRICK", "Z", "S", "H", "CZ_BRICK", "SWAP_BRICK")
    layers, off = [], 0
    for i, k in enumerate(kinds + kinds[::-1]):
        src = "none" if k in fixed else ("input" if i % 5 == 0 else "theta")
        par = i % 2
        cnt = W.layer_param_count(n, (k, src, 0, par))
        layers.append((k, src, 0, par))
    # assign offsets: theta and input counted separately
    b = W._Builder(n)
    for k, src, _, par in layers:
        b.add(k, src, par)
    compare("c64", n, b.layers, 2, seed=5, path=2)


def _fold_circuit(n, name):
    """Leading RX / RY layer followed by a single-qubit layer: the backward
    takes the leading layer's gradients on the next layer's passes."""
    b = W._Builder(n)
    spec = {
        "rx_ry": [("RX", "input"), ("RY", "theta"), ("ISINGZZ_RING", "theta"), ("CNOT_RING", "none"),
                  ("RY", "theta")],
        "ry_rx": [("RY", "input"), ("RX", "theta"), ("CNOT_RING", "none"), ("RX", "theta")],
        "rx_sx": [("RX", "input"), ("SX", "none"), ("RZ", "theta"), ("CNOT_RING", "none"), ("RY", "theta")],
        "ry_gpi2": [("RY", "theta"), ("GPI2", "theta"), ("CNOT_RING", "none"), ("GPI", "theta")],
        "sx_rx_ry": [("SX", "none"), ("RX", "input"), ("RY", "theta"), ("MS_BRICK", "theta")],
    }[name]
    for k, src in spec:
        b.add(k, src)
    return b.layers


@pytest.mark.parametrize("name", ["rx_ry", "ry_rx", "rx_sx", "ry_gpi2", "sx_rx_ry"])
@pytest.mark.parametrize("dtype,n", [("c64", 14), ("c128", 13)])
def test_leading_layer_gradient_folded_into_next_layer(name, dtype, n):
    compare(dtype, n, _fold_circuit(n, name), 3, seed=11, path=2, fuse=1)


def _run_with_env(code, env_extra):
    import os
    import subprocess
    import sys
    env = dict(os.environ, **env_extra)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]


def test_folded_gradients_in_shared_memory_sums():
    """Two register bits per round: more than four rounds per pass, so every
    slot, companions included, keeps its per-thread sums in shared memory
    (defer=2) instead of registers (own process: the knob is read once)."""
    code = ("import sys; sys.path.insert(0, '.');"
            "from tests.test_gpu_parity import compare, _fold_circuit;"
            "[compare('c64', 14, _fold_circuit(14, k), 2, seed=12, path=2) for k in ('rx_ry', 'ry_rx', 'rx_sx')];"
            "compare('c128', 13, _fold_circuit(13, 'ry_gpi2'), 2, seed=12, path=2)")
    _run_with_env(code, {"QC_RB_BWD": "2"})


def test_gradients_reduced_every_round_where_shared_sums_do_not_fit():
    """Complex128 on 2^11-amplitude backward tiles (two buffers): the RX input
    layer's pass has six rounds, and its per-thread sums do not fit in shared
    memory beside two CTAs' tiles, so each round reduces them in FP64
    (defer=0); the plan is checked to take that mode."""
    code = ("import sys; sys.path.insert(0, '.');"
            "from tests.test_gpu_parity import compare;"
            "from paper_2506_04891_gb300 import workloads as W, qlayer as Q;"
            "b = W._Builder(13);"
            "[b.add(k, s, 0) for k, s in (('RX', 'input'), ('ROT', 'theta'), ('CNOT_RING', 'none'), ('ROT', 'theta'))];"
            "d = Q.Circuit(13, b.layers, dtype='c128', path=2).describe(2);"
            "assert any(l.startswith('B') and 'defer=0' in l and 'slots=11' in l for l in d.splitlines()), d;"
            "compare('c128', 13, b.layers, 2, seed=15, path=2)")
    _run_with_env(code, {"QC_TMAX_BWD": "11"})


@pytest.mark.parametrize("rb", [3, 4])
def test_generic_generator_gradient_at_three_and_four_register_bits(rb):
    """GPI2's gradient (a generator that is no Pauli matrix) is summed from
    the anti-Hermitian form of A = M^dagger dM; the backward passes of the
    ionq family run at three and at four register bits (own process: the
    knob is read once), complex64 on TMA tiles and complex128 on per-thread
    copies."""
    code = ("import sys; sys.path.insert(0, '.');"
            "from tests.test_gpu_parity import compare; from paper_2506_04891_gb300 import workloads as W;"
            "compare('c64', 14, W.ionq_circuit(14, 2), 2, seed=21, path=2);"
            "compare('c128', 13, W.ionq_circuit(13, 2), 2, seed=22, path=2)")
    _run_with_env(code, {"QC_RB_BWD": str(rb)})


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("dtype,n", [("c64", 9), ("c128", 8)])
def test_constant_gates_and_rot_both_paths(path, dtype, n):
    """Z, S, H, CZ and SWAP bricks (both parities) and Rot (theta and input
    sourced) around the other kinds (Appendix A matrices)."""
    b = W._Builder(n)
    for k, src, par in [("ROT", "input", 0), ("H", "none", 0), ("CZ_BRICK", "none", 0),
                        ("S", "none", 0), ("RY", "theta", 0), ("SWAP_BRICK", "none", 1),
                        ("Z", "none", 0), ("ROT", "theta", 0), ("CNOT_RING", "none", 0),
                        ("CZ_BRICK", "none", 1), ("SWAP_BRICK", "none", 0), ("ROT", "theta", 0)]:
        b.add(k, src, par)
    compare(dtype, n, b.layers, 3, seed=13, path=path)


@pytest.mark.parametrize("dtype,n,path", [("c64", 14, 2), ("c128", 13, 2), ("c64", 10, 1)])
def test_qdi_reupload_matches_oracle(dtype, n, path):
    """QDI (Sec. 3): the same x re-enters every RZ layer, so several layers add
    into each dx entry."""
    compare(dtype, n, W.qdi_circuit(n, 3), 3, seed=14, path=path)


def test_autotune_picks_a_candidate_and_its_plan_matches_the_oracle():
    from paper_2506_04891_gb300 import tune
    n = 16
    layers = W.ibm_circuit(n, 2)
    r = tune.autotune(n, layers, 2, fwd_candidates=[dict(tile_bits_fwd=12, reg_bits_fwd=4),
                                                    dict(tile_bits_fwd=10, reg_bits_fwd=3)],
                      bwd_candidates=[dict(tile_bits_bwd=11, reg_bits_bwd=3),
                                      dict(tile_bits_bwd=9, reg_bits_bwd=2)])
    assert len(r["timings"]) == 4 and all(ms > 0 for _, _, ms in r["timings"])
    assert r["tuning"]["tile_bits_fwd"] in (10, 12) and r["tuning"]["tile_bits_bwd"] in (9, 11)
    x, theta, g = W.draw_inputs(n, layers, 2, seed=3)
    ref = oracle_all(n, layers, x, theta, g)
    for tuning in ({}, r["tuning"], dict(tile_bits_fwd=9, tile_bits_bwd=8, reg_bits_fwd=2,
                                         reg_bits_bwd=1, stages_fwd=3, stages_bwd=1)):
        import torch
        from paper_2506_04891_gb300 import qlayer as Q
        c = Q.Circuit(n, layers, path=2, tuning=tuning)
        xt = torch.tensor(x, device="cuda")
        tt = torch.tensor(theta, device="cuda")
        ps, ez = c.forward(xt, tt, batch=2)
        dth, dx = c.backward(xt, tt, ps, torch.tensor(g, device="cuda"))
        check("c64", "ez", ez.cpu().numpy(), ref["ez"])
        check("c64", "dx", dx.cpu().numpy(), ref["dx"])
        check("c64", "dtheta", dth.cpu().numpy(), ref["dth"], batch_sum=2)


def test_empty_circuit_and_batch_one():
    for path in (1, 2):
        got = run_gpu(5, [], np.zeros((1, 0)), np.zeros(0), np.full((1, 5), 0.2), dtype="c128", path=path)
        psi = np.zeros(32)
        psi[0] = 1
        assert np.array_equal(got["psi"][0], psi)
        assert np.allclose(got["ez"], 1.0)


def test_random_upstream_gradient():
    n = 9
    layers = W.ionq_circuit(n, 3)
    g = W.draw_upstream(3, n, seed=9)
    compare("c128", n, layers, 3, seed=6, path=2, g=g)
    compare("c128", n, layers, 3, seed=6, path=1, g=g)


# ---------------------------------------------------------------------------
# permutation layers are bit-exact
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,path", [(5, 1), (12, 1), (13, 2), (16, 2), (18, 2)])
@pytest.mark.parametrize("perm", [["CNOT_RING"], ["X"], ["CNOT_RING", "CNOT_RING", "X"]])
def test_permutation_layers_bit_exact(n, path, perm):
    pre = [("RX", "input", 0, 0), ("RY", "theta", 0, 0), ("RZ", "theta", n, 0)]
    x, theta, g = W.draw_inputs(n, pre, 2, seed=7)
    a = run_gpu(n, pre, x, theta, g, path=path, fuse=0)
    b = run_gpu(n, pre + [(k, "none", 0, 0) for k in perm], x, theta, g, path=path, fuse=0)
    # apply the oracle's permutation (exact on any values) to the GPU input state
    exp = np.stack([O.forward_sample(n, [(k, "none", 0, 0) for k in perm], None, None, psi0=a["psi"][i])
                    for i in range(2)])
    assert np.array_equal(b["psi"], exp)


# ---------------------------------------------------------------------------
# properties
# ---------------------------------------------------------------------------

def test_backward_is_deterministic():
    n = 15
    layers = W.ionq_circuit(n, 2)
    x, theta, g = W.draw_inputs(n, layers, 3, seed=8)
    a = run_gpu(n, layers, x, theta, g, path=2)
    b = run_gpu(n, layers, x, theta, g, path=2)
    assert np.array_equal(a["dth"], b["dth"]) and np.array_equal(a["dx"], b["dx"])
    assert np.array_equal(a["ez"], b["ez"])


def test_errors_are_reported_not_raised_on_device():
    import torch
    from paper_2506_04891_gb300 import qlayer as Q
    c = Q.Circuit(14, W.hea_circuit(14, 1), dtype="c64", path=2)
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    x = torch.zeros((2, 14), dtype=torch.float64, device="cuda")
    th = torch.zeros(c.n_theta, dtype=torch.float64, device="cuda")
    with pytest.raises(Q.QCError) as e:
        c.forward(x, th, workspace=small)
    assert e.value.status == 2
    ckc = Q.Circuit(14, W.hea_circuit(14, 2), dtype="c64", path=2, ckpt_every=2)
    xb = torch.zeros((2, ckc.n_in), dtype=torch.float64, device="cuda")
    tb = torch.zeros(ckc.n_theta, dtype=torch.float64, device="cuda")
    psi, _ = ckc.forward(xb, tb)
    other = torch.empty(ckc.workspace_bytes(2) + 4096, dtype=torch.uint8, device="cuda")
    with pytest.raises(Q.QCError) as e:
        ckc.backward(xb, tb, psi, torch.ones((2, 14), dtype=torch.float64, device="cuda"), workspace=other)
    assert e.value.status == 1
    torch.cuda.synchronize()


def test_qc_wait_and_step_host():
    import ctypes
    import torch
    from paper_2506_04891_gb300 import qlayer as Q
    n = 10
    layers = W.zz_circuit(n, 2)
    x, theta, g = W.draw_inputs(n, layers, 4, seed=10)
    c = Q.Circuit(n, layers, dtype="c128", path=2)
    ws = c.workspace(4)
    psi = torch.empty((4, 1 << n), dtype=torch.complex128, device="cuda")
    stg = torch.empty(Q.qc_staging_bytes(c.handle, 4), dtype=torch.uint8, device="cuda")
    xh, th, gh = (np.ascontiguousarray(a) for a in (x, theta, g))
    ez = np.zeros((4, n))
    dth = np.zeros(c.n_theta)
    dx = np.zeros((4, c.n_in))
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p).value  # noqa: E731
    stream = torch.cuda.current_stream().cuda_stream
    Q.qc_step_host(c.handle, 4, P(xh), P(th), P(gh), P(ez), P(dth), P(dx), psi.data_ptr(),
                   ws.data_ptr(), ws.numel(), stg.data_ptr(), stream)
    Q.qc_wait(stream, 10000)
    ref = oracle_all(n, layers, x, theta, g)
    check("c128", "ez", ez, ref["ez"])
    check("c128", "dtheta", dth, ref["dth"])
    check("c128", "dx", dx, ref["dx"])

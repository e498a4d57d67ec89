"""Host-side checks of the C ABI and the planner (no GPU needed).

qc_create, qc_num_params, qc_workspace_bytes and qc_describe_plan never touch
the device, so the library loads and plans on a machine without a GPU.
"""
import os
import re

import pytest

from paper_2506_04891_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qlayer.h")


@pytest.fixture(scope="module")
def q():
    from paper_2506_04891_gb300 import build
    if not os.path.exists(build.OUT):
        build.build()
    from paper_2506_04891_gb300 import qlayer
    return qlayer


def header_symbols():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"QC_API\s+[\w\s\*]+?\b(qc_\w+)\s*\(", txt)))


def test_library_exports_every_header_symbol(q):
    import ctypes
    lib = ctypes.CDLL(q.LIB_PATH)
    syms = header_symbols()
    assert len(syms) >= 12
    for s in syms:
        assert hasattr(lib, s), s
    assert set(q.EXPORTED) <= set(syms)


def test_nm_exports_are_extern_c(q):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", q.LIB_PATH], capture_output=True, text=True).stdout
    names = {l.split()[-1] for l in out.splitlines() if " T " in l}
    for s in header_symbols():
        assert s in names, s


def test_version_and_defaults(q):
    assert q.qc_version() == 101
    o = q.qc_default_options()
    assert (o.ckpt_every, o.path, o.fuse) == (-1, 0, 1)


@pytest.mark.parametrize("name", sorted(W.WORKLOADS))
def test_num_params_match_workload_definition(q, name):
    cfg = W.WORKLOADS[name]
    layers = cfg["layers"]()
    h = q.qc_create(cfg["n"], cfg["dtype"], layers)
    try:
        assert q.qc_num_params(h) == W.circuit_params(cfg["n"], layers)
    finally:
        q.qc_destroy(h)


def test_param_counts_from_the_survey(q):
    # P = 8, 360, 320, 548, 624 for the five circuits
    assert W.circuit_params(4, W.WORKLOADS["hea4"]["layers"]())[0] == 8
    assert W.circuit_params(12, W.WORKLOADS["hea12"]["layers"]())[0] == 360
    assert W.circuit_params(20, W.WORKLOADS["ibm20"]["layers"]())[0] == 320
    assert W.circuit_params(20, W.WORKLOADS["ionq20"]["layers"]())[0] == 548
    assert W.circuit_params(26, W.WORKLOADS["zz26"]["layers"]())[0] == 624


@pytest.mark.parametrize("bad,err", [
    (dict(n=0), 1), (dict(n=31), 1),
    (dict(layers=[("CNOT_RING", "theta", 0, 0)]), 1),      # unparametrised with a source
    (dict(n=1, layers=[("CNOT_RING", "none", 0, 0)]), 1),   # ring needs n >= 2
    (dict(layers=[("MS_BRICK", "theta", 0, 2)]), 1),        # parity
    (dict(layers=[("RX", "theta", -1, 0)]), 1),             # offset
    (dict(n=20, path=1), 5),                                # smem path too large
])
def test_create_rejects_invalid(q, bad, err):
    n = bad.get("n", 4)
    layers = bad.get("layers", [("RX", "input", 0, 0)])
    opt = q.qc_default_options()
    opt.path = bad.get("path", 0)
    with pytest.raises(q.QCError) as e:
        q.qc_create(n, "c64", layers, opt)
    assert e.value.status == err
    assert q.qc_last_error()


def test_calls_refuse_empty_or_negative_batch_and_null_buffers_on_the_host(q):
    """Argument checks run before any CUDA call, so they are exercised here
    without a GPU: a batch of 0 or below, or a NULL state or workspace, is
    QC_ERR_INVALID with a message."""
    h = q.qc_create(4, "c64", [("RX", "input", 0, 0), ("RY", "theta", 0, 0)])
    try:
        for batch in (0, -3):
            with pytest.raises(q.QCError) as e:
                q.qc_workspace_bytes(h, batch)
            assert e.value.status == 1
            with pytest.raises(q.QCError) as e:
                q.qc_forward(h, batch, None, None, None, None, None, 0, None)
            assert e.value.status == 1 and "batch" in q.qc_last_error()
            with pytest.raises(q.QCError) as e:
                q.qc_backward(h, batch, None, None, None, None, None, None, None, 0, None)
            assert e.value.status == 1
            with pytest.raises(q.QCError) as e:
                q.qc_expect_z(h, batch, None, None, None)
            assert e.value.status == 1
        with pytest.raises(q.QCError) as e:
            q.qc_forward(h, 2, None, None, None, None, None, 0, None)
        assert e.value.status == 1 and "psi_out" in q.qc_last_error()
        with pytest.raises(q.QCError) as e:
            q.qc_backward(h, 2, None, None, None, None, None, None, None, 0, None)
        assert e.value.status == 1
    finally:
        q.qc_destroy(h)


def test_rot_counts_three_parameters_per_qubit_and_constants_take_no_source(q):
    n = 6
    h = q.qc_create(n, "c64", [("ROT", "theta", 4, 0), ("H", "none", 0, 0), ("ROT", "input", 1, 0)])
    try:
        assert q.qc_num_params(h) == (4 + 3 * n, 1 + 3 * n)
        assert q.qc_num_params(h) == W.circuit_params(n, [("ROT", "theta", 4, 0), ("ROT", "input", 1, 0)])
    finally:
        q.qc_destroy(h)
    for kind in ("Z", "S", "H", "CZ_BRICK", "SWAP_BRICK"):
        with pytest.raises(q.QCError):
            q.qc_create(n, "c64", [(kind, "theta", 0, 0)])
    with pytest.raises(q.QCError):
        q.qc_create(n, "c64", [("SWAP_BRICK", "none", 0, 2)])


def test_tuning_options_shape_the_plan_and_are_validated(q):
    layers = W.zz_circuit(16, 2)
    base = q.Circuit(16, layers, path=2).describe(2)
    tuned = q.Circuit(16, layers, path=2, tuning=dict(tile_bits_fwd=10, tile_bits_bwd=9,
                                                      reg_bits_fwd=3, reg_bits_bwd=2)).describe(2)
    def geo(desc, tag):
        return {(int(d["t"]), int(d["rb"])) for d in
                (dict(re.findall(r"(\w+)=(-?\d+)", l.split("[")[0])) for l in desc.splitlines()
                 if l.startswith(tag) and " TILE " in l)}
    assert geo(base, "F ") == {(12, 4)} and geo(base, "B ") == {(12, 4)}
    assert geo(tuned, "F ") == {(10, 3)} and geo(tuned, "B ") == {(9, 2)}
    for bad in (dict(tile_bits_fwd=14), dict(tile_bits_bwd=13), dict(tile_bits_fwd=5),
                dict(reg_bits_bwd=5), dict(stages_fwd=4), dict(stages_bwd=-1)):
        with pytest.raises(q.QCError):
            q.Circuit(16, layers, tuning=bad)
    with pytest.raises(q.QCError):
        q.Circuit(16, layers, dtype="c128", tuning=dict(tile_bits_bwd=12))
    with pytest.raises(ValueError):
        q.Circuit(16, layers, tuning=dict(tiles=3))


def test_geometry_environment_fills_unset_options_and_is_validated(q, monkeypatch):
    layers = W.zz_circuit(16, 2)

    def geo(desc, tag):
        return {(int(d["t"]), int(d["rb"])) for d in
                (dict(re.findall(r"(\w+)=(-?\d+)", l.split("[")[0])) for l in desc.splitlines()
                 if l.startswith(tag) and " TILE " in l)}
    monkeypatch.setenv("QC_TMAX_BWD", "10")
    monkeypatch.setenv("QC_RB_FWD", "3")
    env = q.Circuit(16, layers, path=2).describe(2)
    assert geo(env, "F ") == {(12, 3)} and geo(env, "B ") == {(10, 4)}
    # an explicit option wins over the environment
    opt = q.Circuit(16, layers, path=2, tuning=dict(tile_bits_bwd=11)).describe(2)
    assert geo(opt, "B ") == {(11, 4)}
    for name, bad in (("QC_RB_BWD", "9"), ("QC_TMAX_FWD", "20"), ("QC_TILE_STAGES", "5")):
        monkeypatch.setenv(name, bad)
        with pytest.raises(q.QCError) as e:
            q.Circuit(16, layers)
        assert e.value.status == 1 and name.split("_")[1] in q.qc_last_error()
        monkeypatch.delenv(name)


def test_backward_gradient_sums_kept_on_chip_per_pass_kind(q):
    """Per-thread FP32 gradient sums stay on the SM across a CTA's tiles:
    in registers for single-qubit passes of at most four rounds (defer=1), in
    shared memory for the MS brick passes (two-qubit ops, three parameters
    each: defer=2); zz26 keeps every pass in registers."""
    desc = q.Circuit(20, W.ionq_circuit(20, 8), path=2).describe(32)
    tiles = [l for l in desc.splitlines() if l.startswith("B") and " TILE " in l]
    brick = [l for l in tiles if ",2q np=3" in l]
    single = [l for l in tiles if ",2q" not in l]
    assert brick and single
    assert all("defer=2" in l for l in brick)
    assert all("defer=1" in l for l in single)
    zz = q.Circuit(26, W.zz_circuit(26, 12), path=2).describe(8)
    assert all("defer=1" in l for l in zz.splitlines() if l.startswith("B") and " TILE " in l)


def test_forward_diagonal_rides_on_the_contiguous_pass_run_last(q):
    """zz26: each block's IsingZZ phase (but the first, which the product-state
    kernel takes) is multiplied in the last round of the contiguous 2^12 pass,
    which the planner runs last in its group (post=2: compile-time element
    patterns); the gathering pass stays first."""
    desc = q.Circuit(26, W.zz_circuit(26, 12), path=2).describe(8)
    fwd = [dict(re.findall(r"(\w+)=(-?\d+)", l.split("[")[0])) for l in desc.splitlines()
           if l.startswith("F ") and " TILE " in l]
    posts = [d for d in fwd if d["post"] != "0"]
    assert len(posts) == 11 and all(d["post"] == "2" and d["c"] == "12" and d["t"] == "12" for d in posts)
    groups = {}
    for d in fwd:
        groups.setdefault(d["layer"], []).append(d)
    for g in groups.values():
        assert [d["post"] for d in g] == ["0", "0", "2"] and g[0]["h0"] == "19"
    # complex128 (2^11 tiles) keeps the generic last-round phase on the last pass
    d128 = q.Circuit(20, W.zz_circuit(20, 3), dtype="c128", path=2).describe(2)
    assert "post=2" not in d128 and "post=1" in d128


def test_tuner_candidates_stay_in_range():
    from paper_2506_04891_gb300 import tune
    for dtype in ("c64", "c128"):
        fwd, bwd = tune.candidates(26, dtype)
        fm, bm = tune.MAX_TILE[dtype]
        assert fwd and bwd
        assert all(6 <= c["tile_bits_fwd"] <= fm and c["reg_bits_fwd"] in (3, 4) for c in fwd)
        assert all(6 <= c["tile_bits_bwd"] <= bm and 1 <= c["reg_bits_bwd"] <= 4 for c in bwd)
        assert tune.DEFAULT_TILE[dtype][0] in {c["tile_bits_fwd"] for c in fwd}
    fwd, _ = tune.candidates(9, "c64")
    assert all(c["tile_bits_fwd"] <= 9 for c in fwd)


def test_unknown_kind_rejected(q):
    import ctypes
    arr = (q.qc_layer * 1)()
    arr[0] = q.qc_layer(99, 0, 0, 0)
    h = ctypes.c_void_p()
    assert q._lib.qc_create(4, 0, arr, 1, None, ctypes.byref(h)) == 1
    assert h.value is None


def _plan(q, n, layers, dtype="c64", batch=4, path=2, ckpt=-1, fuse=1, **tuning):
    opt = q.qc_default_options()
    opt.path = path
    opt.ckpt_every = ckpt
    opt.fuse = fuse
    for k, v in tuning.items():
        setattr(opt, k, v)
    h = q.qc_create(n, dtype, layers, opt)
    try:
        return q.qc_describe_plan(h, batch), q.qc_workspace_bytes(h, batch)
    finally:
        q.qc_destroy(h)


def _tile_passes(desc):
    out = []
    for line in desc.splitlines():
        if " TILE " not in line:
            continue
        d = dict(re.findall(r"(\w+)=(-?\d+)", line.split("[")[0]))
        ops = re.findall(r"\[l=(\d+)(,2q)? np=(\d+)[^\]]*\]", line)
        out.append((line[0], int(d["layer"]), {k: int(v) for k, v in d.items()}, ops))
    return out


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [5, 11, 12, 13, 14, 17, 20, 23, 26])
@pytest.mark.parametrize("rb", [0, 1, 2, 4])
def test_tile_passes_cover_every_qubit_once(q, n, dtype, rb):
    layers = [("RY", "theta", 0, 0), ("MS_BRICK", "theta", n, 0), ("ECR_BRICK", "none", 0, 1),
              ("RX", "theta", 0, 0)]
    desc, _ = _plan(q, n, layers, dtype=dtype, fuse=0, reg_bits_fwd=rb, reg_bits_bwd=rb)
    tmax = 12 if dtype == "c64" else 11
    for tag in "FB":
        covered = {}
        for t_, layer, d, ops in _tile_passes(desc):
            if t_ != tag:
                continue
            assert d["t"] <= tmax and d["t"] >= 1
            c, h0, t = d["c"], d["h0"], d["t"]
            for l, is2q, np_ in ops:
                l = int(l)
                glob = l if l < c else h0 + (l - c)
                bits = [glob, glob + 1] if is2q else [glob]
                if is2q:
                    # both bits of a brick pair sit in the same range of the tile
                    assert (l + 1 < c) or (l >= c), (layer, l, c)
                for b in bits:
                    key = (layer, b)
                    assert key not in covered, (tag, layer, b)
                    covered[key] = True
        for layer, kind in enumerate(["RY", "MS", "ECR", "RX"]):
            bits = {b for (l_, b) in covered if l_ == layer}
            if kind in ("RY", "RX"):
                assert bits == set(range(n)), (tag, layer)
            elif kind == "MS":
                assert bits == {b for q0 in range(0, n - 1, 2) for b in (n - 2 - q0, n - 1 - q0)}
            else:
                assert bits == {b for q0 in range(1, n - 1, 2) for b in (n - 2 - q0, n - 1 - q0)}


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [5, 12, 13, 17, 20, 26])
@pytest.mark.parametrize("family", ["zz", "hea", "ibm", "ionq", "qdi"])
def test_fused_tile_groups_cover_every_qubit_once(q, family, n, dtype):
    """With fusion on (diagonals as phases, rings as gathers and scatters,
    companion gradients, the contiguous pass moved last for a forward post
    phase, register bits by gate type), each tile group of the plan still
    applies its layer's gates on every bit exactly once; a post phase with
    compile-time patterns sits on a contiguous 2^12 pass that runs last."""
    build = {"zz": W.zz_circuit, "hea": W.hea_circuit, "ibm": W.ibm_circuit,
             "ionq": W.ionq_circuit, "qdi": W.qdi_circuit}[family]
    desc, _ = _plan(q, n, build(n, 3), dtype=dtype)
    groups = []
    for tag, layer, d, ops in _tile_passes(desc):
        if groups and groups[-1][0] == (tag, layer):
            groups[-1][1].append((d, ops))
        else:
            groups.append(((tag, layer), [(d, ops)]))
    assert groups
    for (tag, layer), passes in groups:
        bits = []
        two = False
        for d, ops in passes:
            c, h0 = d["c"], d["h0"]
            for l, is2q, _np in ops:
                l = int(l)
                glob = l if l < c else h0 + (l - c)
                bits += [glob, glob + 1] if is2q else [glob]
                two = two or bool(is2q)
        assert len(bits) == len(set(bits)), (tag, layer, sorted(bits))
        if two:
            assert len(bits) in (2 * ((n - 0) // 2), 2 * ((n - 1) // 2))
        else:
            assert set(bits) == set(range(n)), (tag, layer, sorted(bits))
        for k, (d, _ops) in enumerate(passes):
            if d.get("post") == 2:
                assert k == len(passes) - 1 and d["c"] == d["t"] == 12 and dtype == "c64"


@pytest.mark.parametrize("n", [2, 3, 4, 5, 7, 8])
def test_ring_pair_identity_the_permuted_stores_rely_on(n):
    """The backward ring kernel and the scatter pass store 16-byte pairs because
    the inverse CNOT-ring map sends k and k ^ 1 ^ 2^(n-1) to adjacent indices:
    f^-1(k ^ 1 ^ 2^(n-1)) = f^-1(k) ^ 1.  Checked against the oracle's ring
    layer applied to every basis state."""
    import numpy as np
    from oracle import qsim_oracle as O
    N = 1 << n
    f = np.empty(N, dtype=np.int64)
    for k in range(N):
        e = np.zeros(N, dtype=np.complex128)
        e[k] = 1.0
        out = O.forward_sample(n, [("CNOT_RING", "none", 0, 0)], None, None, psi0=e)
        f[k] = int(np.argmax(np.abs(out)))
        assert abs(out[f[k]]) == 1.0
    finv = np.empty(N, dtype=np.int64)
    finv[f] = np.arange(N)
    top = 1 << (n - 1)
    for k in range(N):
        assert finv[k ^ 1 ^ top] == finv[k] ^ 1, (n, k)


def test_zz26_plan_checkpoints_and_workspace(q):
    cfg = W.WORKLOADS["zz26"]
    desc, ws = _plan(q, 26, cfg["layers"](), batch=8, path=0)
    head = desc.splitlines()[0]
    assert "path=layer" in head and "nlead=2" in head
    nck = int(re.search(r"nckpt=(\d+)", head).group(1))
    assert 4 <= nck <= 9
    S = 8 * 2 ** 26 * 8
    # 2 psi + 2 lambda running buffers + checkpoints, plus gradient partials
    assert (4 + nck) * S <= ws < (4 + nck) * S + 3 * 2 ** 30


def test_fused_zz26_plan_has_no_standalone_ring_or_diag_in_the_forward(q):
    cfg = W.WORKLOADS["zz26"]
    desc, _ = _plan(q, 26, cfg["layers"](), batch=8, path=0)
    fwd = [l for l in desc.splitlines() if l.startswith("F ")]
    assert sum(" RING " in l for l in fwd) == 1      # the final ring only
    assert not any(" DIAG " in l for l in fwd)
    assert sum(" TILE " in l for l in fwd) == 11 * 3
    # checkpoints hold states that the backward re-reads (diagonal-layer inputs)
    bwd = [l for l in desc.splitlines() if l.startswith("B ")]
    assert sum(" RING " in l for l in bwd) == 1      # the last ring (lambda formed there)
    assert not any("LAMINIT" in l for l in bwd)


def test_leading_rotation_layer_folds_into_the_next_backward_layer(q):
    """RX(x) then RY(theta): the embedding's gradients ride on the RY passes
    (companion X slots), so the backward never undoes layer 0 and the last RY
    pass skips its store; without fusion layer 0 gets its own passes."""
    cfg = W.WORKLOADS["zz26"]
    desc, _ = _plan(q, 26, cfg["layers"](), batch=8, path=0)
    bwd = [l for l in desc.splitlines() if l.startswith("B ")]
    assert not any(l.startswith("B layer=0 ") for l in bwd)
    l1 = [l for l in bwd if l.startswith("B layer=1 TILE")]
    assert len(l1) == 3
    nops = sum(int(re.search(r" ops=(\d+)", l).group(1)) for l in l1)
    assert nops == 26 and sum(l.count("+X") for l in l1) == 26
    for l in l1:
        d = dict(re.findall(r"(\w+)=(-?\d+)", l.split("[")[0]))
        assert int(d["slots"]) == 2 * int(d["ops"])
    assert "store=0" in l1[-1] and all("store=1" in l for l in l1[:-1])
    plain, _ = _plan(q, 26, cfg["layers"](), batch=8, path=0, fuse=0)
    assert any(l.startswith("B layer=0 TILE") for l in plain.splitlines())
    assert "+X" not in plain
    # a parameter-free single-qubit layer carries only companion slots
    b = W._Builder(14)
    b.add("RY", "input")
    b.add("SX")
    b.add("RZ", "theta")
    sx, _ = _plan(q, 14, b.layers)
    for l in sx.splitlines():
        if l.startswith("B layer=1 TILE"):
            assert "+Y" in l and " np=1" not in l
    # not folded when an earlier layer still needs the backward sweep
    b = W._Builder(14)
    b.add("RZ", "theta")
    b.add("RX", "input")
    b.add("RY", "theta")
    mid, _ = _plan(q, 14, b.layers)
    assert "+X" not in mid and any(l.startswith("B layer=1 TILE") for l in mid.splitlines())


def test_backward_diagonal_layers_ride_in_the_next_tile_pass(q):
    """zz26 backward: each IsingZZ ring layer is undone (and differentiated)
    in round 0 of the next RY layer's contiguous pass, so no standalone
    diagonal pass is left; without fusion every one is its own pass."""
    cfg = W.WORKLOADS["zz26"]
    desc, _ = _plan(q, 26, cfg["layers"](), batch=8, path=0)
    bwd = [l for l in desc.splitlines() if l.startswith("B ")]
    assert not any(" DIAG " in l for l in bwd)
    pre = [l for l in bwd if "pre=1" in l]
    assert len(pre) == 12
    for l in pre:
        d = dict(re.findall(r"(\w+)=(-?\d+)", l.split("[")[0]))
        assert d["c"] == d["t"] and int(d["t"]) - int(d["rb"]) <= 8
    plain, _ = _plan(q, 26, cfg["layers"](), batch=8, path=0, fuse=0)
    assert sum(" DIAG " in l for l in plain.splitlines() if l.startswith("B ")) == 12
    assert "pre=1" not in plain


def test_backward_diagonal_before_a_ring_rides_in_the_ring_pass(q):
    """HEA blocks [RZ, RY, RZ, CNOT ring]: in the backward the first RZ of a
    block is undone (and differentiated) in the tiled ring pass that follows
    it, so no standalone diagonal pass is left; with fusion off it is one."""
    layers = W.serving_circuit(24)
    desc, _ = _plan(q, 24, layers, batch=2, path=2)
    bwd = [l for l in desc.splitlines() if l.startswith("B ")]
    assert not any(" DIAG " in l for l in bwd)
    assert sum(" RING " in l and "pre=1" in l for l in bwd) == 5
    plain, _ = _plan(q, 24, layers, batch=2, path=2, fuse=0)
    assert sum(" DIAG " in l for l in plain.splitlines() if l.startswith("B ")) >= 6


def test_x_layers_ride_in_complemented_loads_out_of_place(q):
    """ibm20: every X layer of the body is applied (forward, the brick's
    first pass) and undone (backward, the SX pass) by loading tile k from ~k;
    such a pass reads another CTA's tile, so it never writes in place."""
    cfg = W.WORKLOADS["ibm20"]
    desc, _ = _plan(q, cfg["n"], cfg["layers"](), batch=cfg["batch"], path=2)
    xl = [l for l in desc.splitlines() if " xl=1 " in l]
    assert sum(l.startswith("F ") for l in xl) == 7 and sum(l.startswith("B ") for l in xl) == 8
    for l in xl:
        d = dict(re.findall(r"(\w+)=(-?\d+)", l.split("[")[0]))
        assert d["src"] != d["dst"] and d["tma"] == "1", l
    assert not any(" DIAG " in l and "xcomp=1" in l for l in desc.splitlines())


def test_automatic_path_takes_shared_memory_only_where_launch_bound(q):
    """The whole-circuit shared-memory kernel for small states (hea4, and
    n <= 10 / n <= 8 at batch <= 128), the layer path above (hea12 in both
    precisions measured 1.5-1.6x faster on it)."""
    expect = {"hea4": True, "hea12": False, "hea12_c128": False}
    for name, smem in expect.items():
        cfg = W.WORKLOADS[name]
        desc, _ = _plan(q, cfg["n"], cfg["layers"](), dtype=cfg["dtype"], batch=cfg["batch"], path=0)
        assert ("path=smem" in desc.splitlines()[0]) == smem, (name, desc.splitlines()[0])
    for n, dtype, B, smem in [(10, "c64", 64, True), (10, "c64", 256, False), (11, "c64", 1, False),
                              (8, "c128", 128, True), (9, "c128", 4, False)]:
        desc, _ = _plan(q, n, W.serving_circuit(n), dtype=dtype, batch=B, path=0)
        assert ("path=smem" in desc.splitlines()[0]) == smem, (n, dtype, B)


def test_forward_plan_ends_in_psi_out(q):
    for name in ("ibm20", "ionq20", "zz26"):
        cfg = W.WORKLOADS[name]
        desc, _ = _plan(q, cfg["n"], cfg["layers"](), batch=cfg["batch"], path=0)
        fwd = [l for l in desc.splitlines() if l.startswith("F ")]
        last = dict(re.findall(r"(\w+)=(-?\d+)", fwd[-1].split("[")[0]))
        assert last["dst"] == "0", fwd[-1]
        # no forward step writes into a buffer it reads unless it is an in-place kind
        for line in fwd:
            if " RING " in line:
                d = dict(re.findall(r"(\w+)=(-?\d+)", line))
                assert d["src"] != d["dst"]


def test_backward_never_writes_psi_out(q):
    for name in ("ibm20", "zz26"):
        cfg = W.WORKLOADS[name]
        desc, _ = _plan(q, cfg["n"], cfg["layers"](), batch=cfg["batch"], path=0)
        for line in desc.splitlines():
            if line.startswith("B ") and "dst=" in line:
                d = dict(re.findall(r"(\w+)=(-?\d+)", line))
                assert d["dst"] != "0", line


def test_workspace_grows_with_batch(q):
    layers = W.hea_circuit(14, 2)
    _, w1 = _plan(q, 14, layers, batch=1)
    _, w8 = _plan(q, 14, layers, batch=8)
    assert w8 > w1 > 0


def test_planning_many_batches_allocates_nothing_and_keeps_tables_in_the_workspace(q):
    """Plans are host-only: sizing and describing plans for many batch sizes
    (more than the handle keeps) makes no device allocation, frees nothing and
    never synchronises, and the workspace holds the plan tables."""
    layers = W.hea_circuit(16, 2)
    c = q.Circuit(16, layers, dtype="c64", path=2)
    a0 = q.qc_alloc_count()
    sizes = {}
    for b in list(range(1, 41)) + [7, 3, 1]:
        sizes[b] = c.workspace_bytes(b)
        assert "TILE" in c.describe(b)
    assert q.qc_alloc_count() == a0
    # a plan rebuilt after it left the bounded cache has the same layout
    assert c.workspace_bytes(1) == sizes[1] and c.workspace_bytes(40) == sizes[40]
    assert sizes[40] > sizes[1]

"""Plain, slow CPU oracle for layered QML state-vector simulation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  The CUDA library never calls it and shares no code with it.

Everything here is complex128 numpy, one sample at a time, one gate at a time:

* gate matrices follow the paper's Appendix A ("Matrix Representations"), with
  two printed matrices corrected (MS and ECR are not unitary as printed; see
  ``ms`` and ``ECR`` below for the reading used);
* a layer is expanded into its individual gates and each gate is applied by
  Einstein summation over the gate's qubit axes of the state reshaped to
  ``[2]*n`` (Sec. 2.2.2, "Sequential Einsum"); qubit 0 is axis 0, i.e. the most
  significant bit of the flat index (the binary counting matrix J of Sec. 2.4.1
  lists qubit 0 in its first column);
* <Z_q> = sum_k |psi_k|^2 (1 - 2 b_q(k)) (measurement of single-qubit Z, Sec. 3);
* gradients: a per-gate reverse sweep (adjoint method) with the analytic
  derivative of every gate matrix; parameter-shift and central finite
  differences are provided to pin it.

Layer description (shared plain structure, no arithmetic): a tuple
``(kind, source, offset, parity)`` where ``kind`` is one of ``LAYER_KINDS``,
``source`` is ``"theta"`` (trainable vector shared by the batch), ``"input"``
(per-sample data x[b]) or ``"none"`` (all parameters zero / unparametrised),
``offset`` is the index of the layer's first parameter in theta or x[b], and
``parity`` (0 or 1) selects the brick pattern of two-qubit brick layers.

Parameters per layer:
* RX, RY, RZ, GPI, GPI2: n (parameter j acts on qubit j);
* ROT: 3n, qubit j reads (theta, phi, lambda) = parameters 3j, 3j+1, 3j+2 of the
  matrix Rot(theta, phi, lambda) printed in Appendix A;
* ISINGZZ_RING: n (parameter j acts on the pair (j, (j+1) mod n), Sec. 2.4.1
  formula for K_Rzz; for n = 2 this is the same pair twice);
* MS_BRICK: 3 per gate (phi0, phi1, theta), gate i on qubits
  (parity + 2i, parity + 2i + 1), no wrap-around;
* CNOT_RING, X, SX, ECR_BRICK, Z, S, H, CZ_BRICK, SWAP_BRICK: none (Z, S, H
  on every qubit; CZ and SWAP on the brick pairs).
CNOT_RING applies CNOT(q -> q+1 mod n) for q = 0, 1, ..., n-1 in that order.

Angles of GPI, GPI2 and MS are in turns, as printed in Appendix A
(exp(2 pi i phi), cos(pi theta)).
"""
from __future__ import annotations

import numpy as np

LAYER_KINDS = (
    "RX", "RY", "RZ", "ISINGZZ_RING", "CNOT_RING", "X", "SX",
    "GPI", "GPI2", "MS_BRICK", "ECR_BRICK",
    "Z", "S", "H", "CZ_BRICK", "SWAP_BRICK", "ROT",
)

# ---------------------------------------------------------------------------
# Gate matrices (Appendix A)
# ---------------------------------------------------------------------------
I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
S = np.array([[1, 0], [0, 1j]], dtype=np.complex128)
H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2.0)
SX = 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]], dtype=np.complex128)
CNOT = np.array([[1, 0, 0, 0],
                 [0, 1, 0, 0],
                 [0, 0, 0, 1],
                 [0, 0, 1, 0]], dtype=np.complex128)
CZ = np.diag([1, 1, 1, -1]).astype(np.complex128)
SWAP = np.array([[1, 0, 0, 0],
                 [0, 0, 1, 0],
                 [0, 1, 0, 0],
                 [0, 0, 0, 1]], dtype=np.complex128)
# ECR as printed (Appendix A) has rows 1-2 = (0,1,0,i), (1,0,-i,0) / sqrt(2) but
# rows 3-4 that make it non-unitary.  Reading used: ECR = (I (x) X - X (x) Y) / sqrt(2)
# with the first qubit the left Kronecker factor, which reproduces the two
# printed rows and is Hermitian, unitary and an involution.
ECR = (np.kron(I2, X) - np.kron(X, Y)) / np.sqrt(2.0)


def rx(t):
    c, s = np.cos(t / 2), np.sin(t / 2)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def ry(t):
    c, s = np.cos(t / 2), np.sin(t / 2)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def rz(t):
    return np.array([[np.exp(-0.5j * t), 0], [0, np.exp(0.5j * t)]], dtype=np.complex128)


def isingzz(t):
    a, b = np.exp(-0.5j * t), np.exp(0.5j * t)
    return np.diag([a, b, b, a]).astype(np.complex128)


def gpi(phi):
    return np.array([[0, np.exp(-2j * np.pi * phi)],
                     [np.exp(2j * np.pi * phi), 0]], dtype=np.complex128)


def gpi2(phi):
    return np.array([[1, -1j * np.exp(-2j * np.pi * phi)],
                     [-1j * np.exp(2j * np.pi * phi), 1]], dtype=np.complex128) / np.sqrt(2.0)


def rot(theta, phi, lam):
    """Rot(theta, phi, lambda) as printed in Appendix A ("Other gates")."""
    c, s = np.cos(theta / 2), np.sin(theta / 2)
    return np.array([[c, -np.exp(1j * lam) * s],
                     [np.exp(1j * phi) * s, np.exp(1j * (phi + lam)) * c]], dtype=np.complex128)


def ms(phi0, phi1, theta):
    """Molmer-Sorensen gate (Appendix A, "Other gates").

    As printed, entries (0,3) and (3,0) carry the same phase, which makes the
    matrix non-unitary.  Reading used: entry (3,0) takes the conjugate phase
    exp(+2 pi i (phi0 + phi1)); the middle block is kept exactly as printed.
    """
    c, s = np.cos(np.pi * theta), np.sin(np.pi * theta)
    m = np.zeros((4, 4), dtype=np.complex128)
    m[0, 0] = m[1, 1] = m[2, 2] = m[3, 3] = c
    m[0, 3] = -1j * np.exp(-2j * np.pi * (phi0 + phi1)) * s
    m[1, 2] = -1j * np.exp(-2j * np.pi * (phi1 - phi0)) * s
    m[2, 1] = -1j * np.exp(-2j * np.pi * (phi0 - phi1)) * s
    m[3, 0] = -1j * np.exp(+2j * np.pi * (phi0 + phi1)) * s
    return m


# Analytic derivatives of the parametrised matrices ------------------------

def d_rx(t):
    c, s = np.cos(t / 2), np.sin(t / 2)
    return 0.5 * np.array([[-s, -1j * c], [-1j * c, -s]], dtype=np.complex128)


def d_ry(t):
    c, s = np.cos(t / 2), np.sin(t / 2)
    return 0.5 * np.array([[-s, -c], [c, -s]], dtype=np.complex128)


def d_rz(t):
    return np.array([[-0.5j * np.exp(-0.5j * t), 0], [0, 0.5j * np.exp(0.5j * t)]],
                    dtype=np.complex128)


def d_isingzz(t):
    a, b = -0.5j * np.exp(-0.5j * t), 0.5j * np.exp(0.5j * t)
    return np.diag([a, b, b, a]).astype(np.complex128)


def d_gpi(phi):
    w = 2j * np.pi
    return np.array([[0, -w * np.exp(-w * phi)], [w * np.exp(w * phi), 0]], dtype=np.complex128)


def d_gpi2(phi):
    w = 2j * np.pi
    return np.array([[0, -1j * (-w) * np.exp(-w * phi)],
                     [-1j * w * np.exp(w * phi), 0]], dtype=np.complex128) / np.sqrt(2.0)


def d_rot(theta, phi, lam):
    """Partial derivatives (d/dtheta, d/dphi, d/dlambda) of ``rot``."""
    c, s = np.cos(theta / 2), np.sin(theta / 2)
    el, ep, epl = np.exp(1j * lam), np.exp(1j * phi), np.exp(1j * (phi + lam))
    dth = 0.5 * np.array([[-s, -el * c], [ep * c, -epl * s]], dtype=np.complex128)
    dph = np.array([[0, 0], [1j * ep * s, 1j * epl * c]], dtype=np.complex128)
    dla = np.array([[0, -1j * el * s], [0, 1j * epl * c]], dtype=np.complex128)
    return dth, dph, dla


def d_ms(phi0, phi1, theta):
    """Partial derivatives (d/dphi0, d/dphi1, d/dtheta) of ``ms``."""
    c, s = np.cos(np.pi * theta), np.sin(np.pi * theta)
    w = 2j * np.pi
    e03 = np.exp(-w * (phi0 + phi1))
    e12 = np.exp(-w * (phi1 - phi0))
    e21 = np.exp(-w * (phi0 - phi1))
    e30 = np.exp(+w * (phi0 + phi1))
    dphi0 = np.zeros((4, 4), dtype=np.complex128)
    dphi1 = np.zeros((4, 4), dtype=np.complex128)
    dth = np.zeros((4, 4), dtype=np.complex128)
    # d/dphi0
    dphi0[0, 3] = -1j * s * (-w) * e03
    dphi0[1, 2] = -1j * s * (+w) * e12
    dphi0[2, 1] = -1j * s * (-w) * e21
    dphi0[3, 0] = -1j * s * (+w) * e30
    # d/dphi1
    dphi1[0, 3] = -1j * s * (-w) * e03
    dphi1[1, 2] = -1j * s * (-w) * e12
    dphi1[2, 1] = -1j * s * (+w) * e21
    dphi1[3, 0] = -1j * s * (+w) * e30
    # d/dtheta
    ds = np.pi * c
    dc = -np.pi * s
    for k in range(4):
        dth[k, k] = dc
    dth[0, 3] = -1j * e03 * ds
    dth[1, 2] = -1j * e12 * ds
    dth[2, 1] = -1j * e21 * ds
    dth[3, 0] = -1j * e30 * ds
    return dphi0, dphi1, dth


# ---------------------------------------------------------------------------
# Layers -> gates
# ---------------------------------------------------------------------------

def layer_num_params(n, kind):
    """Number of parameters a layer of ``kind`` on n qubits reads."""
    if kind in ("RX", "RY", "RZ", "GPI", "GPI2", "ISINGZZ_RING"):
        return n
    if kind == "ROT":
        return 3 * n
    if kind == "MS_BRICK":
        raise ValueError("MS_BRICK parameter count depends on parity; use brick_pairs")
    return 0


def brick_pairs(n, parity):
    """Qubit pairs of a brick layer: (parity + 2i, parity + 2i + 1), no wrap."""
    return [(q, q + 1) for q in range(parity, n - 1, 2)]


def layer_param_count(n, layer):
    kind, _source, _offset, parity = layer
    if kind == "MS_BRICK":
        return 3 * len(brick_pairs(n, parity))
    return layer_num_params(n, kind)


def _param_value(layer, j, x_b, theta):
    _kind, source, offset, _parity = layer
    if source == "theta":
        return float(theta[offset + j])
    if source == "input":
        return float(x_b[offset + j])
    if source == "none":
        return 0.0
    raise ValueError(f"unknown source {source!r}")


def layer_gates(n, layer, x_b, theta):
    """Expand one layer into gates.

    Returns a list of (qubits, matrix, derivs) where ``derivs`` is a list of
    (source, index, dmatrix) for every trainable/differentiable parameter of the
    gate (``index`` is the position in theta or x[b]).
    """
    kind, source, offset, parity = layer
    gates = []
    diff = source in ("theta", "input")

    def ref(j):
        return (source, offset + j) if diff else None

    if kind in ("RX", "RY", "RZ", "GPI", "GPI2"):
        fn, dfn = {"RX": (rx, d_rx), "RY": (ry, d_ry), "RZ": (rz, d_rz),
                   "GPI": (gpi, d_gpi), "GPI2": (gpi2, d_gpi2)}[kind]
        for q in range(n):
            t = _param_value(layer, q, x_b, theta)
            derivs = [(ref(q)[0], ref(q)[1], dfn(t))] if diff else []
            gates.append(((q,), fn(t), derivs))
    elif kind == "ISINGZZ_RING":
        if n < 2:
            raise ValueError("ring layers need n >= 2")
        for j in range(n):
            t = _param_value(layer, j, x_b, theta)
            derivs = [(ref(j)[0], ref(j)[1], d_isingzz(t))] if diff else []
            gates.append(((j, (j + 1) % n), isingzz(t), derivs))
    elif kind == "CNOT_RING":
        if n < 2:
            raise ValueError("ring layers need n >= 2")
        for q in range(n):
            gates.append(((q, (q + 1) % n), CNOT, []))
    elif kind == "X":
        for q in range(n):
            gates.append(((q,), X, []))
    elif kind == "SX":
        for q in range(n):
            gates.append(((q,), SX, []))
    elif kind == "ECR_BRICK":
        for pair in brick_pairs(n, parity):
            gates.append((pair, ECR, []))
    elif kind in ("Z", "S", "H"):
        U = {"Z": Z, "S": S, "H": H}[kind]
        for q in range(n):
            gates.append(((q,), U, []))
    elif kind in ("CZ_BRICK", "SWAP_BRICK"):
        U = CZ if kind == "CZ_BRICK" else SWAP
        for pair in brick_pairs(n, parity):
            gates.append((pair, U, []))
    elif kind == "ROT":
        for q in range(n):
            th = _param_value(layer, 3 * q + 0, x_b, theta)
            ph = _param_value(layer, 3 * q + 1, x_b, theta)
            la = _param_value(layer, 3 * q + 2, x_b, theta)
            derivs = []
            if diff:
                dth, dph, dla = d_rot(th, ph, la)
                derivs = [(source, offset + 3 * q + 0, dth),
                          (source, offset + 3 * q + 1, dph),
                          (source, offset + 3 * q + 2, dla)]
            gates.append(((q,), rot(th, ph, la), derivs))
    elif kind == "MS_BRICK":
        for i, pair in enumerate(brick_pairs(n, parity)):
            p0 = _param_value(layer, 3 * i + 0, x_b, theta)
            p1 = _param_value(layer, 3 * i + 1, x_b, theta)
            th = _param_value(layer, 3 * i + 2, x_b, theta)
            derivs = []
            if diff:
                d0, d1, d2 = d_ms(p0, p1, th)
                derivs = [(source, offset + 3 * i + 0, d0),
                          (source, offset + 3 * i + 1, d1),
                          (source, offset + 3 * i + 2, d2)]
            gates.append((pair, ms(p0, p1, th), derivs))
    else:
        raise ValueError(f"unknown layer kind {kind!r}")
    return gates


# ---------------------------------------------------------------------------
# State-vector primitives (Sequential Einsum, Sec. 2.2.2)
# ---------------------------------------------------------------------------

def apply_local(psi_t, U, qubits):
    """psi'_{..i'_k..i'_m..} = U^{i'_k i'_m}_{i_k i_m} psi_{..i_k..i_m..}.

    ``psi_t`` has shape [2]*n; ``U`` is a 2^l x 2^l matrix on ``qubits``
    (first qubit = most significant index of U).
    """
    n = psi_t.ndim
    l = len(qubits)
    Ut = U.reshape([2] * (2 * l))
    # contract U's input indices (last l axes) with the state's qubit axes
    out = np.tensordot(Ut, psi_t, axes=(list(range(l, 2 * l)), list(qubits)))
    # out axes: U's output indices (l), then the remaining state axes in order
    rest = [a for a in range(n) if a not in qubits]
    order = list(qubits) + rest
    inv = np.argsort(order)
    return np.transpose(out, inv)


def zero_state(n):
    psi = np.zeros(2 ** n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def forward_sample(n, layers, x_b, theta, psi0=None):
    """psi_L = U_L ... U_1 |0...0> for one sample (complex128, flat 2^n)."""
    psi = zero_state(n) if psi0 is None else np.array(psi0, dtype=np.complex128)
    psi_t = psi.reshape([2] * n)
    for layer in layers:
        for qubits, U, _ in layer_gates(n, layer, x_b, theta):
            psi_t = apply_local(psi_t, U, qubits)
    return psi_t.reshape(-1)


def forward(n, layers, x, theta):
    """Batched forward: x has shape [B, n_in]; returns [B, 2^n] complex128."""
    return np.stack([forward_sample(n, layers, x[b], theta) for b in range(x.shape[0])])


def expect_z_sample(psi, n):
    """<Z_q> for q = 0..n-1 of one flat state."""
    p = (np.abs(psi) ** 2).reshape([2] * n)
    out = np.empty(n)
    for q in range(n):
        axes = tuple(a for a in range(n) if a != q)
        m = p.sum(axis=axes)
        out[q] = m[0] - m[1]
    return out


def expect_z(psi_batch, n):
    return np.stack([expect_z_sample(psi_batch[b], n) for b in range(psi_batch.shape[0])])


def z_observable_diag(n, g):
    """Diagonal of O = sum_q g_q Z_q as a [2]*n tensor."""
    d = np.zeros([2] * n)
    for q in range(n):
        shape = [1] * n
        shape[q] = 2
        d = d + g[q] * np.array([1.0, -1.0]).reshape(shape)
    return d


def adjoint_sample(n, layers, x_b, theta, g_b, n_theta, n_in):
    """Reverse-sweep adjoint gradient of L = sum_q g_q <Z_q> for one sample.

    Returns (ez[n], dtheta[n_theta], dx[n_in]).  For every gate U with
    parameter p: dL/dp = 2 Re <lambda_after| dU |psi_before>, where
    psi_before = U^dagger psi_after and lambda is propagated backwards by U^dagger,
    starting from lambda_L = O psi_L.
    """
    psi_t = forward_sample(n, layers, x_b, theta).reshape([2] * n)
    ez = expect_z_sample(psi_t.reshape(-1), n)
    lam_t = z_observable_diag(n, g_b) * psi_t
    dtheta = np.zeros(n_theta)
    dx = np.zeros(n_in)
    gate_list = []
    for layer in layers:
        gate_list.extend(layer_gates(n, layer, x_b, theta))
    for qubits, U, derivs in reversed(gate_list):
        Ud = U.conj().T
        psi_before = apply_local(psi_t, Ud, qubits)
        for source, idx, dU in derivs:
            v = apply_local(psi_before, dU, qubits)
            g = 2.0 * np.real(np.vdot(lam_t.reshape(-1), v.reshape(-1)))
            if source == "theta":
                dtheta[idx] += g
            else:
                dx[idx] += g
        lam_t = apply_local(lam_t, Ud, qubits)
        psi_t = psi_before
    return ez, dtheta, dx


def num_params(n, layers):
    """(n_theta, n_input_per_sample) read by a circuit."""
    n_theta = 0
    n_in = 0
    for layer in layers:
        c = layer_param_count(n, layer)
        if c == 0:
            continue
        _k, source, offset, _p = layer
        if source == "theta":
            n_theta = max(n_theta, offset + c)
        elif source == "input":
            n_in = max(n_in, offset + c)
    return n_theta, n_in


def adjoint(n, layers, x, theta, g):
    """Batched adjoint: returns (ez[B,n], dtheta[P] summed over the batch,
    dtheta_per_sample[B,P], dx[B,n_in])."""
    n_theta, n_in = num_params(n, layers)
    n_theta = max(n_theta, len(theta))
    n_in = max(n_in, x.shape[1] if x.ndim == 2 else 0)
    B = x.shape[0]
    ez = np.zeros((B, n))
    dth = np.zeros((B, n_theta))
    dx = np.zeros((B, n_in))
    for b in range(B):
        ez[b], dth[b], dx[b] = adjoint_sample(n, layers, x[b], theta, g[b], n_theta, n_in)
    return ez, dth.sum(axis=0), dth, dx


# ---------------------------------------------------------------------------
# Independent gradient rules used to pin the adjoint
# ---------------------------------------------------------------------------

def loss_sample(n, layers, x_b, theta, g_b):
    psi = forward_sample(n, layers, x_b, theta)
    return float(np.dot(g_b, expect_z_sample(psi, n)))


def finite_diff_sample(n, layers, x_b, theta, g_b, h=1e-6):
    """Central finite differences of sum_q g_q <Z_q> w.r.t. theta and x_b."""
    theta = np.array(theta, dtype=np.float64)
    x_b = np.array(x_b, dtype=np.float64)
    dth = np.zeros_like(theta)
    dx = np.zeros_like(x_b)
    for i in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        dth[i] = (loss_sample(n, layers, x_b, tp, g_b) - loss_sample(n, layers, x_b, tm, g_b)) / (2 * h)
    for i in range(x_b.size):
        xp, xm = x_b.copy(), x_b.copy()
        xp[i] += h
        xm[i] -= h
        dx[i] = (loss_sample(n, layers, xp, theta, g_b) - loss_sample(n, layers, xm, theta, g_b)) / (2 * h)
    return dth, dx


# Exact two-term shift rules: a parameter entering as exp(-i a p K) with K^2 = I
# has df/dp = a [f(p + pi/(4a)) - f(p - pi/(4a))].
#   RX, RY, RZ, IsingZZ: a = 1/2  -> shift pi/2,  factor 1/2
#   MS theta (exp(-i pi theta K)):  a = pi  -> shift 1/4, factor pi
#   GPI phi (exp(-2 pi i phi Z) X up to the order of factors): a = 2 pi -> shift 1/8
SHIFT_RULES = {
    "RX": (np.pi / 2, 0.5), "RY": (np.pi / 2, 0.5), "RZ": (np.pi / 2, 0.5),
    "ISINGZZ_RING": (np.pi / 2, 0.5),
    "GPI": (0.125, 2 * np.pi),
    "MS_THETA": (0.25, np.pi),
    # Rot: theta enters as RY(theta); phi and lambda through a phase e^{i a}
    # on one basis state, a generator with eigenvalues 0 and 1
    "ROT": (np.pi / 2, 0.5),
}


def param_shift_sample(n, layers, x_b, theta, g_b):
    """Parameter-shift gradient for every parameter whose rule is exact.

    Returns dict {(source, index): value}.  Every parameter of a layer is used
    by exactly one gate in the circuits considered, so shifting the stored
    value shifts exactly one gate.
    """
    out = {}
    theta = np.array(theta, dtype=np.float64)
    x_b = np.array(x_b, dtype=np.float64)
    for layer in layers:
        kind, source, offset, parity = layer
        if source not in ("theta", "input"):
            continue
        idxs = []
        if kind in SHIFT_RULES:
            idxs = [(offset + j, SHIFT_RULES[kind]) for j in range(layer_param_count(n, layer))]
        elif kind == "MS_BRICK":
            idxs = [(offset + 3 * i + 2, SHIFT_RULES["MS_THETA"])
                    for i in range(len(brick_pairs(n, parity)))]
        for idx, (shift, factor) in idxs:
            vec = theta if source == "theta" else x_b
            vp, vm = vec.copy(), vec.copy()
            vp[idx] += shift
            vm[idx] -= shift
            if source == "theta":
                fp = loss_sample(n, layers, x_b, vp, g_b)
                fm = loss_sample(n, layers, x_b, vm, g_b)
            else:
                fp = loss_sample(n, layers, vp, theta, g_b)
                fm = loss_sample(n, layers, vm, theta, g_b)
            out[(source, idx)] = out.get((source, idx), 0.0) + factor * (fp - fm)
    return out


# ---------------------------------------------------------------------------
# Brute force (Unitary operation, Sec. 2.2.1): whole-layer 2^n x 2^n matrices
# ---------------------------------------------------------------------------

def full_gate_matrix(n, U, qubits):
    """2^n x 2^n matrix of a local gate, built from Kronecker products and an
    explicit basis permutation (no einsum)."""
    l = len(qubits)
    N = 2 ** n
    M = np.zeros((N, N), dtype=np.complex128)
    for col in range(N):
        bits = [(col >> (n - 1 - q)) & 1 for q in range(n)]
        sub_in = 0
        for q in qubits:
            sub_in = (sub_in << 1) | bits[q]
        for sub_out in range(2 ** l):
            amp = U[sub_out, sub_in]
            if amp == 0:
                continue
            nb = list(bits)
            for i, q in enumerate(qubits):
                nb[q] = (sub_out >> (l - 1 - i)) & 1
            row = 0
            for b in nb:
                row = (row << 1) | b
            M[row, col] += amp
    return M


def kron_layer_matrix(n, gates_1q):
    """Kronecker product of per-qubit 2x2 matrices (qubit 0 leftmost)."""
    M = np.array([[1.0 + 0j]])
    for U in gates_1q:
        M = np.kron(M, U)
    return M


def layer_unitary(n, layer, x_b, theta):
    """2^n x 2^n matrix of a whole layer (product of its gate matrices)."""
    M = np.eye(2 ** n, dtype=np.complex128)
    for qubits, U, _ in layer_gates(n, layer, x_b, theta):
        M = full_gate_matrix(n, U, qubits) @ M
    return M


def forward_bruteforce(n, layers, x_b, theta):
    psi = zero_state(n)
    for layer in layers:
        psi = layer_unitary(n, layer, x_b, theta) @ psi
    return psi


# ---------------------------------------------------------------------------
# Diagonal layers: Eigenphase Computation and Diagonal Tensor Product (Sec. 2.4)
# ---------------------------------------------------------------------------

def binary_counting_matrix(n):
    """J: 2^n x n, row i = binary digits of i, most significant first."""
    return np.array([[(i >> (n - 1 - j)) & 1 for j in range(n)] for i in range(2 ** n)],
                    dtype=np.int64)


def k_rz(n):
    """K_Rz = 1 - 2 J (entries +1 for bit 0, -1 for bit 1)."""
    return 1 - 2 * binary_counting_matrix(n)


def k_rzz_ring(n):
    """K_Rzz[i, j] = K_Rz[i, j] * K_Rz[i, (j + 1) mod n]."""
    K = k_rz(n)
    return K * K[:, [(j + 1) % n for j in range(n)]]


def ec_diagonal(K, theta):
    """Eigenphase Computation.  The printed exp(i K theta) disagrees with the
    printed Rz matrix diag(e^{-i theta/2}, e^{i theta/2}); the reading used is
    alpha = -(1/2) K theta, which reproduces the Rz / Rzz matrices."""
    return np.exp(-0.5j * (K @ np.asarray(theta, dtype=np.float64)))


def tp_diagonal(diags_1q):
    """Diagonal Tensor Product: diag(U) = kron_i diag(U^(i))."""
    d = np.array([1.0 + 0j])
    for v in diags_1q:
        d = np.kron(d, v)
    return d

"""Circuit structures and seeded synthetic inputs of the benchmark workloads.

This module holds no simulation arithmetic: it only lists layers (as plain
``(kind, source, offset, parity)`` tuples) and draws seeded random inputs.  It
is the one module that both the CUDA path's callers and the oracle's callers
share.

Workloads (the paper's circuits are synthetic with random inputs, Sec. 3):

* ``hea4``   n=4,  B=8,   RX(x) embedding, 2 x [RY(theta), CNOT ring]
* ``hea12``  n=12, B=256, RX(x) embedding, 10 x [RZ, RY, RZ, CNOT ring]
* ``ibm20``  n=20, B=32,  SX, RZ(x) encoding, 8 x [RZ, SX, RZ, X, ECR brick]
* ``ionq20`` n=20, B=32,  GPI2(0), RZ(x) encoding, 8 x [GPI, GPI2, MS brick]
* ``zz26``   n=26, B=8,   RX(x) embedding, 12 x [RY, IsingZZ ring, CNOT ring]
* serving requests: RX(x), 6 x [RZ, RY, RZ, CNOT ring], n in 8..24, B in 1..512
  (``serve20`` / ``serve24``: that circuit at n = 20 and 24 with B = 2)

The native-gate bodies (IBM: ECR, X, SX, RZ; IonQ: GPI, GPI2, MS with a
virtual-RZ encoding layer) follow the gate sets named in Appendix B; the
exact ordering inside the repeated block is not printed (the circuit figure is
not available) and is the reading stated above.  Brick parity alternates with
block depth d (d mod 2).

Draws: numpy ``default_rng(seed)``; x ~ U[0, pi) and theta ~ U[0, 2 pi) in
float64.  IonQ/IBM angles are drawn the same way and passed as printed
(GPI/GPI2/MS take turns), so every gate still sweeps whole periods.
"""
from __future__ import annotations

import math

import numpy as np

PARAM_KINDS_N = ("RX", "RY", "RZ", "GPI", "GPI2", "ISINGZZ_RING")


def brick_gate_count(n: int, parity: int) -> int:
    """Number of pairs (parity + 2i, parity + 2i + 1) with no wrap-around."""
    return max(0, (n - parity) // 2)


def layer_param_count(n: int, layer) -> int:
    kind, _s, _o, parity = layer
    if kind in PARAM_KINDS_N:
        return n
    if kind == "MS_BRICK":
        return 3 * brick_gate_count(n, parity)
    if kind == "ROT":
        return 3 * n
    return 0


class _Builder:
    def __init__(self, n: int):
        self.n = n
        self.layers = []
        self.n_theta = 0
        self.n_in = 0

    def add(self, kind: str, source: str = "none", parity: int = 0):
        cnt = layer_param_count(self.n, (kind, source, 0, parity))
        if source == "theta":
            off = self.n_theta
            self.n_theta += cnt
        elif source == "input":
            off = self.n_in
            self.n_in += cnt
        else:
            off = 0
        self.layers.append((kind, source, off, parity))


def hea_circuit(n: int, depth: int, block=("RZ", "RY", "RZ"), embed="RX"):
    """Hardware-efficient ansatz: embedding layer, then depth x [trainable
    rotation layers + CNOT ring]."""
    b = _Builder(n)
    b.add(embed, "input")
    for _ in range(depth):
        for k in block:
            b.add(k, "theta")
        b.add("CNOT_RING")
    return b.layers


def qdi_circuit(n: int, depth: int):
    """Quantum Depth Infused layer (Sec. 3): the data x re-enters in every RZ
    layer (the same n inputs each block), between trainable RY / RZ layers and a
    CNOT ring."""
    b = _Builder(n)
    for _ in range(depth):
        b.layers.append(("RZ", "input", 0, 0))
        b.n_in = max(b.n_in, n)
        b.add("RY", "theta")
        b.add("RZ", "theta")
        b.add("CNOT_RING")
    return b.layers


def zz_circuit(n: int, depth: int):
    b = _Builder(n)
    b.add("RX", "input")
    for _ in range(depth):
        b.add("RY", "theta")
        b.add("ISINGZZ_RING", "theta")
        b.add("CNOT_RING")
    return b.layers


def ibm_circuit(n: int, depth: int = 8):
    b = _Builder(n)
    b.add("SX")
    b.add("RZ", "input")
    for d in range(depth):
        b.add("RZ", "theta")
        b.add("SX")
        b.add("RZ", "theta")
        b.add("X")
        b.add("ECR_BRICK", parity=d % 2)
    return b.layers


def ionq_circuit(n: int, depth: int = 8):
    b = _Builder(n)
    b.add("GPI2")  # GPI2(0): unparametrised, phase 0
    b.add("RZ", "input")
    for d in range(depth):
        b.add("GPI", "theta")
        b.add("GPI2", "theta")
        b.add("MS_BRICK", "theta", parity=d % 2)
    return b.layers


WORKLOADS = {
    "hea4": dict(n=4, batch=8, dtype="c128",
                 layers=lambda: hea_circuit(4, 2, block=("RY",))),
    "hea12": dict(n=12, batch=256, dtype="c64", layers=lambda: hea_circuit(12, 10)),
    "hea12_c128": dict(n=12, batch=256, dtype="c128", layers=lambda: hea_circuit(12, 10)),
    "ibm20": dict(n=20, batch=32, dtype="c64", layers=lambda: ibm_circuit(20, 8)),
    "ionq20": dict(n=20, batch=32, dtype="c64", layers=lambda: ionq_circuit(20, 8)),
    "zz26": dict(n=26, batch=8, dtype="c64", layers=lambda: zz_circuit(26, 12)),
    # the serving request circuit at the two largest qubit counts of the stream
    "serve20": dict(n=20, batch=2, dtype="c64", layers=lambda: serving_circuit(20)),
    "serve24": dict(n=24, batch=2, dtype="c64", layers=lambda: serving_circuit(24)),
}


def circuit_params(n: int, layers):
    """(n_theta, n_input_per_sample) of a layer list."""
    n_theta = n_in = 0
    for layer in layers:
        kind, source, off, parity = layer
        c = layer_param_count(n, layer)
        if source == "theta":
            n_theta = max(n_theta, off + c)
        elif source == "input":
            n_in = max(n_in, off + c)
    return n_theta, n_in


def draw_inputs(n: int, layers, batch: int, seed: int = 0):
    """Seeded x[B, n_in] ~ U[0, pi), theta[P] ~ U[0, 2 pi), and the upstream
    gradient g[B, n] = 1/n (d loss / d <Z_q> for the mean of <Z>)."""
    n_theta, n_in = circuit_params(n, layers)
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, math.pi, size=(batch, n_in))
    theta = rng.uniform(0.0, 2.0 * math.pi, size=(n_theta,))
    g = np.full((batch, n), 1.0 / n)
    return x, theta, g


def draw_upstream(batch: int, n: int, seed: int = 0):
    """Random upstream gradient (used where a non-uniform G is wanted)."""
    rng = np.random.default_rng(seed + 7919)
    return rng.uniform(-1.0, 1.0, size=(batch, n))


def serving_requests(count: int, seed: int = 0, n_range=(8, 24), b_range=(1, 512)):
    """Seeded serving stream: list of (n, batch) pairs, uniform in the ranges."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_range[0], n_range[1] + 1, size=count)
    bs = rng.integers(b_range[0], b_range[1] + 1, size=count)
    return list(zip(ns.tolist(), bs.tolist()))


def serving_circuit(n: int):
    return hea_circuit(n, 6)

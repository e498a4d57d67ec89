"""Host-side checks of the algebra the backward kernels rely on (no GPU).

* Generic single-qubit gradients: the kernels sum 2 Re <w|A|y> over a thread's
  amplitude pairs, A = M^dagger dM, in a reduced form that holds because A is
  anti-Hermitian for a unitary M:
      2 Re <w|A|y> = 2 Re(A01 D) - 2 a0 Im(w0* y0) - 2 a1 Im(w1* y1),
      A00 = i a0, A11 = i a1, D = w0* y1 - w1 conj(y0),
  with D and the two imaginary parts built from six componentwise (packed)
  products per pair.  Checked for every parametrised single-qubit gate of the
  oracle (its matrices and analytic derivatives).
* End-of-pass gradient sums: each value is summed over a warp's 32 lanes in
  FP32 by a butterfly before the FP64 sums across warps; the butterfly's
  error stays within 5 * 2^-24 of the summed magnitudes.
"""
import numpy as np
import pytest

from oracle import qsim_oracle as O

RNG = np.random.default_rng(20506)


def _gates():
    """(name, M, dM) for every parametrised single-qubit gate, at random angles."""
    out = []
    for _ in range(4):
        t = RNG.uniform(-2 * np.pi, 2 * np.pi)
        out += [("rx", O.rx(t), O.d_rx(t)), ("ry", O.ry(t), O.d_ry(t)), ("rz", O.rz(t), O.d_rz(t))]
        phi = RNG.uniform(0, 1)
        out += [("gpi", O.gpi(phi), O.d_gpi(phi)), ("gpi2", O.gpi2(phi), O.d_gpi2(phi))]
        th, ph, la = RNG.uniform(0, 2 * np.pi, 3)
        for k, d in enumerate(O.d_rot(th, ph, la)):
            out.append((f"rot_d{k}", O.rot(th, ph, la), d))
    return out


@pytest.mark.parametrize("name,M,dM", _gates())
def test_generator_is_anti_hermitian(name, M, dM):
    A = M.conj().T @ dM
    assert np.abs(A + A.conj().T).max() < 1e-12, name


def _reduced(A, w, y):
    a0, a1, a01 = A[0, 0].imag, A[1, 1].imag, A[0, 1]
    imq00 = np.sum(np.imag(np.conj(w[:, 0]) * y[:, 0]))
    imq11 = np.sum(np.imag(np.conj(w[:, 1]) * y[:, 1]))
    D = np.sum(np.conj(w[:, 0]) * y[:, 1] - w[:, 1] * np.conj(y[:, 0]))
    return 2 * np.real(a01 * D) - 2 * a0 * imq00 - 2 * a1 * imq11


def _packed(A, w, y):
    """The kernels' six packed accumulators, restated componentwise."""
    sw = lambda z: np.stack([z.imag, z.real], -1)   # (y.y, y.x)
    pr = lambda z: np.stack([z.real, z.imag], -1)   # (y.x, y.y)
    w0, w1, y0, y1 = pr(w[:, 0]), pr(w[:, 1]), y[:, 0], y[:, 1]
    pa = np.sum(w0 * pr(y1), 0)
    pb = np.sum(w1 * pr(y0), 0)
    pc = np.sum(w0 * sw(y1), 0)
    pd = np.sum(w1 * sw(y0), 0)
    pe = np.sum(w0 * sw(y0), 0)
    pf = np.sum(w1 * sw(y1), 0)
    dre = (pa[0] + pa[1]) - (pb[0] + pb[1])
    dim = (pc[0] - pc[1]) + (pd[0] - pd[1])
    a0, a1, a01 = A[0, 0].imag, A[1, 1].imag, A[0, 1]
    return 2 * (a01.real * dre - a01.imag * dim) - 2 * (a0 * (pe[0] - pe[1]) + a1 * (pf[0] - pf[1]))


@pytest.mark.parametrize("name,M,dM", _gates())
def test_reduced_gradient_form_matches_the_definition(name, M, dM):
    A = M.conj().T @ dM
    w = RNG.normal(size=(8, 2)) + 1j * RNG.normal(size=(8, 2))
    y = RNG.normal(size=(8, 2)) + 1j * RNG.normal(size=(8, 2))
    ref = sum(2 * np.real(w[k].conj() @ A @ y[k]) for k in range(8))
    scale = np.abs(A).max() * np.abs(w).max() * np.abs(y).max() * 8
    assert abs(_reduced(A, w, y) - ref) < 1e-12 * scale, name
    assert abs(_packed(A, w, y) - ref) < 1e-12 * scale, name


def test_a_planted_non_anti_hermitian_generator_breaks_the_reduced_form():
    """The reduced form uses only Im A00, Im A11 and A01: a generator with a
    real diagonal part or A10 != -conj(A01) is not covered, so the form must
    disagree with the definition there (guards against a test that cannot fail)."""
    A = np.array([[0.3 + 1.0j, 0.2 - 0.5j], [0.7 + 0.1j, -0.4j]])
    w = RNG.normal(size=(8, 2)) + 1j * RNG.normal(size=(8, 2))
    y = RNG.normal(size=(8, 2)) + 1j * RNG.normal(size=(8, 2))
    ref = sum(2 * np.real(w[k].conj() @ A @ y[k]) for k in range(8))
    assert abs(_reduced(A, w, y) - ref) > 1e-3


def test_fp32_warp_butterfly_error_bound():
    """32 lanes summed by five xor-butterfly levels in FP32 (every lane ends
    with the total; lane 0's is kept) against the FP64 sum."""
    for trial in range(200):
        x = (RNG.normal(size=32) * 10.0 ** RNG.uniform(-3, 3, 32)).astype(np.float32)
        v = x.copy()
        for o in (16, 8, 4, 2, 1):
            v = (v + v[np.arange(32) ^ o]).astype(np.float32)
        exact = np.sum(x.astype(np.float64))
        assert abs(float(v[0]) - exact) <= 5 * 2.0 ** -24 * np.sum(np.abs(x.astype(np.float64))) * (1 + 1e-6)

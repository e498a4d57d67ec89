"""Thin Python binding of the C ABI in include/qlayer.h.

Argument marshalling only: every step of the simulation runs in the CUDA
library ``libqlayer.so`` built in-tree by ``paper_2506_04891_gb300.build``.
Importing this module loads that library and raises if it is missing; there
is no CPU fallback.

Two levels:

* ``qc_*`` functions with the same names and arguments as the C ABI (device
  pointers are Python ints);
* ``Circuit``, which owns a handle and works with torch CUDA tensors (torch
  supplies device memory and the current stream).
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqlayer.so")

KINDS = {
    "RX": 0, "RY": 1, "RZ": 2, "ISINGZZ_RING": 3, "CNOT_RING": 4, "X": 5, "SX": 6,
    "GPI": 7, "GPI2": 8, "MS_BRICK": 9, "ECR_BRICK": 10,
    "Z": 11, "S": 12, "H": 13, "CZ_BRICK": 14, "SWAP_BRICK": 15, "ROT": 16,
}
SOURCES = {"none": 0, "theta": 1, "input": 2}
DTYPES = {"c64": 0, "c128": 1}
STATUS = {0: "QC_OK", 1: "QC_ERR_INVALID", 2: "QC_ERR_OOM", 3: "QC_ERR_CUDA", 4: "QC_ERR_TIMEOUT",
          5: "QC_ERR_UNSUPPORTED"}

# Symbols include/qlayer.h declares (checked by the tests).
EXPORTED = [
    "qc_version", "qc_default_options", "qc_create", "qc_destroy", "qc_num_params",
    "qc_workspace_bytes", "qc_forward", "qc_expect_z", "qc_expect_z_noalloc", "qc_backward",
    "qc_staging_bytes",
    "qc_step_host", "qc_wait", "qc_last_error", "qc_launch_count", "qc_alloc_count",
    "qc_kernel_timeouts",
    "qc_profile_enable",
    "qc_profile_summary", "qc_describe_plan", "qc_fma_peak",
]


class qc_layer(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("source", ctypes.c_int32),
                ("offset", ctypes.c_int32), ("parity", ctypes.c_int32)]


class qc_options(ctypes.Structure):
    _fields_ = [("ckpt_every", ctypes.c_int32), ("path", ctypes.c_int32),
                ("fuse", ctypes.c_int32), ("tile_bits_fwd", ctypes.c_int32),
                ("tile_bits_bwd", ctypes.c_int32), ("reg_bits_fwd", ctypes.c_int32),
                ("reg_bits_bwd", ctypes.c_int32), ("stages_fwd", ctypes.c_int32),
                ("stages_bwd", ctypes.c_int32), ("tma", ctypes.c_int32), ("tc_dense", ctypes.c_int32)]

TUNING_FIELDS = ("tile_bits_fwd", "tile_bits_bwd", "reg_bits_fwd", "reg_bits_bwd", "stages_fwd",
                 "stages_bwd", "tma", "tc_dense")


class QCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -m paper_2506_04891_gb300.build` "
            "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    I = ctypes.c_int
    S = ctypes.c_size_t
    sig = {
        "qc_version": (I, []),
        "qc_default_options": (None, [ctypes.POINTER(qc_options)]),
        "qc_create": (I, [I, I, ctypes.POINTER(qc_layer), I, ctypes.POINTER(qc_options),
                          ctypes.POINTER(P)]),
        "qc_destroy": (I, [P]),
        "qc_num_params": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "qc_workspace_bytes": (I, [P, I, ctypes.POINTER(S)]),
        "qc_forward": (I, [P, I, P, P, P, P, P, S, P]),
        "qc_expect_z": (I, [P, I, P, P, P]),
        "qc_expect_z_noalloc": (I, [P, I, P, P, P]),
        "qc_backward": (I, [P, I, P, P, P, P, P, P, P, S, P]),
        "qc_staging_bytes": (I, [P, I, ctypes.POINTER(S)]),
        "qc_step_host": (I, [P, I, P, P, P, P, P, P, P, P, S, P, P]),
        "qc_wait": (I, [P, I]),
        "qc_last_error": (ctypes.c_char_p, []),
        "qc_describe_plan": (I, [P, I, ctypes.c_char_p, S]),
        "qc_launch_count": (ctypes.c_ulonglong, []),
        "qc_alloc_count": (ctypes.c_ulonglong, []),
        "qc_kernel_timeouts": (I, [ctypes.POINTER(ctypes.c_ulonglong)]),
        "qc_profile_enable": (I, [I]),
        "qc_profile_summary": (I, [ctypes.c_char_p, S]),
        "qc_fma_peak": (I, [I, ctypes.POINTER(ctypes.c_double)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def _check(status: int):
    if status != 0:
        raise QCError(status, _lib.qc_last_error().decode())


# ---------------------------------------------------------------------------
# C-ABI-named wrappers (pointers are ints)
# ---------------------------------------------------------------------------

def qc_version() -> int:
    return _lib.qc_version()


def qc_default_options() -> qc_options:
    o = qc_options()
    _lib.qc_default_options(ctypes.byref(o))
    return o


def make_layers(layers):
    arr = (qc_layer * max(len(layers), 1))()
    for i, (kind, source, offset, parity) in enumerate(layers):
        arr[i] = qc_layer(KINDS[kind], SOURCES[source], int(offset), int(parity))
    return arr


def qc_create(n: int, dtype: str, layers, opt: qc_options | None = None) -> int:
    arr = make_layers(layers)
    h = ctypes.c_void_p()
    _check(_lib.qc_create(int(n), DTYPES[dtype], arr, len(layers),
                          ctypes.byref(opt) if opt is not None else None, ctypes.byref(h)))
    return h.value


def qc_destroy(h: int):
    _check(_lib.qc_destroy(h))


def qc_num_params(h: int):
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(_lib.qc_num_params(h, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def qc_workspace_bytes(h: int, batch: int) -> int:
    v = ctypes.c_size_t()
    _check(_lib.qc_workspace_bytes(h, int(batch), ctypes.byref(v)))
    return v.value


def qc_staging_bytes(h: int, batch: int) -> int:
    v = ctypes.c_size_t()
    _check(_lib.qc_staging_bytes(h, int(batch), ctypes.byref(v)))
    return v.value


def qc_forward(h, batch, x, theta, psi_out, ez, workspace, workspace_bytes, stream):
    _check(_lib.qc_forward(h, int(batch), x, theta, psi_out, ez, workspace, workspace_bytes, stream))


def qc_expect_z(h, batch, psi, ez, stream):
    _check(_lib.qc_expect_z(h, int(batch), psi, ez, stream))


def qc_expect_z_noalloc(h, batch, psi, ez, stream):
    """<Z> without any device allocation (partial sums in the library's fixed
    device array; see include/qlayer.h for the limit and the ordering rule)."""
    _check(_lib.qc_expect_z_noalloc(h, int(batch), psi, ez, stream))


def qc_backward(h, batch, x, theta, psi_out, g_ez, d_theta, d_x, workspace, workspace_bytes, stream):
    _check(_lib.qc_backward(h, int(batch), x, theta, psi_out, g_ez, d_theta, d_x, workspace,
                            workspace_bytes, stream))


def qc_step_host(h, batch, x_h, th_h, g_h, ez_h, dth_h, dx_h, psi_out, workspace, wbytes, staging,
                 stream):
    _check(_lib.qc_step_host(h, int(batch), x_h, th_h, g_h, ez_h, dth_h, dx_h, psi_out, workspace,
                             wbytes, staging, stream))


def qc_wait(stream, timeout_ms: int):
    _check(_lib.qc_wait(stream, int(timeout_ms)))


def qc_last_error() -> str:
    return _lib.qc_last_error().decode()


def qc_launch_count() -> int:
    return _lib.qc_launch_count()


def qc_alloc_count() -> int:
    return _lib.qc_alloc_count()


def qc_kernel_timeouts() -> int:
    """CTAs that gave up waiting for a TMA tile copy since the last call (synchronises)."""
    v = ctypes.c_ulonglong()
    _check(_lib.qc_kernel_timeouts(ctypes.byref(v)))
    return v.value


def qc_profile_enable(on: bool):
    _check(_lib.qc_profile_enable(1 if on else 0))


def qc_profile_summary():
    """{kernel class: (launches, total_ms, algorithmic_bytes)} (synchronises)."""
    buf = ctypes.create_string_buffer(1 << 16)
    _check(_lib.qc_profile_summary(buf, len(buf)))
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms, by = line.split()
        out[name] = (int(cnt), float(ms), float(by))
    return out


def qc_fma_peak(kind: int) -> float:
    """Measured TFLOP/s: 0 FP32 fmaf, 1 FP32x2 FFMA2, 2 FP64 fma (synchronises)."""
    v = ctypes.c_double()
    _check(_lib.qc_fma_peak(int(kind), ctypes.byref(v)))
    return v.value


def qc_describe_plan(h: int, batch: int) -> str:
    buf = ctypes.create_string_buffer(1 << 20)
    _check(_lib.qc_describe_plan(h, int(batch), buf, len(buf)))
    return buf.value.decode()


# ---------------------------------------------------------------------------
# torch-facing wrapper
# ---------------------------------------------------------------------------

def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Circuit:
    """A circuit of uniformly applied layers on n qubits.

    ``layers``: list of (kind, source, offset, parity) tuples (see
    include/qlayer.h); ``dtype``: "c64" or "c128".
    """

    def __init__(self, n: int, layers, dtype: str = "c64", ckpt_every: int = -1, path: int = 0,
                 fuse: int = 1, tuning: dict | None = None):
        self.n = int(n)
        self.layers = list(layers)
        self.dtype = dtype
        opt = qc_default_options()
        opt.ckpt_every = ckpt_every
        opt.path = path
        opt.fuse = fuse
        self.tuning = dict(tuning or {})
        for k, v in self.tuning.items():
            if k not in TUNING_FIELDS:
                raise ValueError(f"unknown tuning field {k!r}")
            setattr(opt, k, int(v))
        self.handle = qc_create(self.n, dtype, self.layers, opt)
        self.n_theta, self.n_in = qc_num_params(self.handle)
        self._ws = {}

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                qc_destroy(h)
            except Exception:
                pass
            self.handle = None

    @property
    def state_dtype(self):
        import torch
        return torch.complex64 if self.dtype == "c64" else torch.complex128

    def workspace_bytes(self, batch: int) -> int:
        return qc_workspace_bytes(self.handle, batch)

    def describe(self, batch: int) -> str:
        return qc_describe_plan(self.handle, batch)

    def uses_checkpoints(self, batch: int) -> bool:
        import re
        m = re.search(r"nckpt=(\d+)", self.describe(batch).splitlines()[0])
        return bool(m and int(m.group(1)) > 0)

    def workspace(self, batch: int, device=None):
        import torch
        ws = self._ws.get(batch)
        if ws is None:
            nb = max(self.workspace_bytes(batch), 256)
            ws = torch.empty(nb, dtype=torch.uint8, device=device or "cuda")
            self._ws = {batch: ws}  # keep one workspace alive
        return ws

    def _prep(self, x, theta, batch):
        import torch
        dev = "cuda"
        if x is not None:
            x = x.to(device=dev, dtype=torch.float64).contiguous()
        if theta is not None:
            theta = theta.to(device=dev, dtype=torch.float64).contiguous()
        return x, theta

    def forward(self, x, theta, batch: int | None = None, psi_out=None, ez=True, stream=None,
                workspace=None):
        """Returns (psi[B, 2^n], ez[B, n] or None)."""
        import torch
        if batch is None:
            batch = x.shape[0] if x is not None else 1
        x, theta = self._prep(x, theta, batch)
        if psi_out is None:
            psi_out = torch.empty((batch, 1 << self.n), dtype=self.state_dtype, device="cuda")
        ez_t = torch.empty((batch, self.n), dtype=torch.float64, device="cuda") if ez else None
        ws = workspace if workspace is not None else self.workspace(batch)
        qc_forward(self.handle, batch, _ptr(x), _ptr(theta), _ptr(psi_out), _ptr(ez_t), _ptr(ws),
                   ws.numel(), _stream_handle(stream))
        return psi_out, ez_t

    def expect_z(self, psi, stream=None):
        import torch
        batch = psi.shape[0]
        ez = torch.empty((batch, self.n), dtype=torch.float64, device="cuda")
        qc_expect_z(self.handle, batch, _ptr(psi), _ptr(ez), _stream_handle(stream))
        return ez

    def backward(self, x, theta, psi_out, g_ez, stream=None, workspace=None, need_dx=True):
        """Returns (d_theta[P], d_x[B, n_in])."""
        import torch
        batch = psi_out.shape[0]
        x, theta = self._prep(x, theta, batch)
        g = g_ez.to(device="cuda", dtype=torch.float64).contiguous()
        dth = torch.empty((max(self.n_theta, 1),), dtype=torch.float64, device="cuda")
        dx = torch.empty((batch, max(self.n_in, 1)), dtype=torch.float64, device="cuda") if need_dx else None
        ws = workspace if workspace is not None else self.workspace(batch)
        qc_backward(self.handle, batch, _ptr(x), _ptr(theta), _ptr(psi_out), _ptr(g), _ptr(dth),
                    _ptr(dx), _ptr(ws), ws.numel(), _stream_handle(stream))
        return dth[: self.n_theta], (dx[:, : self.n_in] if dx is not None else None)

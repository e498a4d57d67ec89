"""Planner tuning on the device.

The layer path's tile geometry (tile bits and register bits per round for the
forward and backward sweeps, shared-memory stages) has defaults that suit the
zz26 workload on a GB300; other circuits, sizes and batches may prefer others.
``autotune`` times candidate geometries through the C ABI on synthetic inputs
of the requested shape and returns the fastest (forward and backward options
are independent, so each sweep is tuned with the other at its default).  The
results never depend on the geometry beyond floating-point rounding.

    from paper_2506_04891_gb300 import tune, workloads as W
    best = tune.autotune(20, W.ibm_circuit(20, 8), batch=32)
    circ = Q.Circuit(20, layers, tuning=best["tuning"])
"""
from __future__ import annotations

import itertools

from . import qlayer as Q
from . import workloads as W

DEFAULT_TILE = {"c64": (12, 12), "c128": (11, 10)}  # (forward, backward) tile bits
MAX_TILE = {"c64": (13, 12), "c128": (12, 11)}


def candidates(n: int, dtype: str):
    """Forward and backward candidate lists around the defaults."""
    f0, b0 = DEFAULT_TILE[dtype]
    fm, bm = MAX_TILE[dtype]
    fwd = [dict(tile_bits_fwd=t, reg_bits_fwd=r, stages_fwd=s)
           for t, r, s in itertools.product([f0 - 1, f0, min(f0 + 1, fm)], [3, 4], [1, 2, 3])
           if t <= n]
    bwd = [dict(tile_bits_bwd=t, reg_bits_bwd=r, stages_bwd=s)
           for t, r, s in itertools.product([b0 - 1, b0, min(b0 + 1, bm)], [2, 3, 4], [1, 2])
           if t <= n]
    # drop duplicates that clamping produced
    dedup = lambda xs: [dict(t) for t in {tuple(sorted(d.items())) for d in xs}]
    return sorted(dedup(fwd), key=lambda d: sorted(d.items())), sorted(dedup(bwd), key=lambda d: sorted(d.items()))


def _time(circ, batch, x, th, g, sweep: str, reps: int, warmup: int):
    import torch
    ws = torch.empty(max(circ.workspace_bytes(batch), 256), dtype=torch.uint8, device="cuda")
    psi = torch.empty((batch, 1 << circ.n), dtype=circ.state_dtype, device="cuda")
    dth = torch.empty((circ.n_theta,), dtype=torch.float64, device="cuda")
    dx = torch.empty((batch, max(circ.n_in, 1)), dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    h = st.cuda_stream

    def fwd():
        Q.qc_forward(circ.handle, batch, x.data_ptr() if x is not None else None,
                     th.data_ptr() if th is not None else None, psi.data_ptr(), None,
                     ws.data_ptr(), ws.numel(), h)

    def bwd():
        Q.qc_backward(circ.handle, batch, x.data_ptr() if x is not None else None,
                      th.data_ptr() if th is not None else None, psi.data_ptr(), g.data_ptr(),
                      dth.data_ptr(), dx.data_ptr(), ws.data_ptr(), ws.numel(), h)

    run = fwd if sweep == "fwd" else bwd
    fwd()
    for _ in range(warmup):
        if sweep == "bwd":
            fwd()
        run()
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(reps):
        if sweep == "bwd":
            fwd()  # backward re-anchors from the forward's checkpoints
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        run()
        b.record(st)
        torch.cuda.synchronize()
        total += a.elapsed_time(b)
    del ws, psi, dth, dx
    return total / reps


def autotune(n: int, layers, batch: int, dtype: str = "c64", reps: int = 2, warmup: int = 1,
             ckpt_every: int = -1, seed: int = 0, fwd_candidates=None, bwd_candidates=None):
    """Times every candidate and returns {"tuning": best options, "fwd_ms",
    "bwd_ms", "timings": [(sweep, options, ms), ...]}."""
    import torch
    fc, bc = candidates(n, dtype)
    fc = fc if fwd_candidates is None else fwd_candidates
    bc = bc if bwd_candidates is None else bwd_candidates
    xn, thn, gn = W.draw_inputs(n, layers, batch, seed=seed)
    x = torch.tensor(xn, dtype=torch.float64, device="cuda") if xn.size else None
    th = torch.tensor(thn, dtype=torch.float64, device="cuda") if thn.size else None
    g = torch.tensor(gn, dtype=torch.float64, device="cuda")
    timings = []
    best = {}
    for sweep, cands in (("fwd", fc), ("bwd", bc)):
        best_ms, best_cfg = None, {}
        for cfg in cands:
            circ = Q.Circuit(n, layers, dtype=dtype, ckpt_every=ckpt_every, path=2, tuning=cfg)
            ms = _time(circ, batch, x, th, g, sweep, reps, warmup)
            del circ
            torch.cuda.empty_cache()
            timings.append((sweep, cfg, ms))
            if best_ms is None or ms < best_ms:
                best_ms, best_cfg = ms, cfg
        best[sweep] = (best_ms, best_cfg)
    tuning = dict(best["fwd"][1])
    tuning.update(best["bwd"][1])
    return {"tuning": tuning, "fwd_ms": best["fwd"][0], "bwd_ms": best["bwd"][0], "timings": timings}


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="zz26", choices=sorted(W.WORKLOADS))
    ap.add_argument("--reps", type=int, default=2)
    a = ap.parse_args()
    cfg = W.WORKLOADS[a.workload]
    r = autotune(cfg["n"], cfg["layers"](), cfg["batch"], cfg["dtype"], reps=a.reps)
    print(json.dumps({"workload": a.workload, **{k: v for k, v in r.items() if k != "timings"},
                      "timings": [[s, c, round(m, 3)] for s, c, m in r["timings"]]}))

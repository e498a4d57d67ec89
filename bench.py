#!/usr/bin/env python3
"""Benchmark of the layered QML simulator: forward + <Z> + adjoint backward.

One JSON line (rank 0).  A step is one fwd+bwd evaluation of the whole
batch: forward through every layer, <Z_q> of every qubit, the adjoint
backward through every layer, and (N > 1) the all-reduce of d theta.

Default workload zz26: n = 26 qubits, batch 8 per GPU, complex64, RX(x)
embedding then 12 x [RY(theta), IsingZZ ring(theta), CNOT ring] (37 layers,
624 trainable angles); every state pass moves 4 GiB per state, far more than
L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2506_04891_gb300 import workloads as W  # noqa: E402

METRIC = "fwd+bwd circuit evals/s"
UNIT = "evals/s"
DESCR = {
    "zz26": "zz26: n=26, batch 8/GPU, complex64; RX(x) + 12x[RY, IsingZZ ring, CNOT ring]; fwd + <Z> + adjoint bwd",
    "hea12": "hea12: n=12, batch 256/GPU, complex64; RX(x) + 10x[RZ, RY, RZ, CNOT ring]; fwd + <Z> + adjoint bwd",
    "ibm20": "ibm20: n=20, batch 32/GPU, complex64; IBM native body depth 8; fwd + <Z> + adjoint bwd",
    "ionq20": "ionq20: n=20, batch 32/GPU, complex64; IonQ native body depth 8; fwd + <Z> + adjoint bwd",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="zz26", choices=sorted(DESCR))
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-budget", type=float, default=15.0, help=argparse.SUPPRESS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    # smaller cases of the same circuit family, for profiling captures
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--batch", type=int, default=None)
    ap.add_argument("--depth", type=int, default=None)
    return ap.parse_args()


def workload_cfg(args):
    cfg = dict(W.WORKLOADS[args.workload])
    if args.n is None and args.batch is None and args.depth is None:
        return cfg, DESCR[args.workload]
    n = args.n or cfg["n"]
    B = args.batch or cfg["batch"]
    fam = {"zz26": lambda d: W.zz_circuit(n, d or 12), "hea12": lambda d: W.hea_circuit(n, d or 10),
           "ibm20": lambda d: W.ibm_circuit(n, d or 8), "ionq20": lambda d: W.ionq_circuit(n, d or 8)}
    layers = fam[args.workload](args.depth)
    cfg.update(n=n, batch=B, layers=lambda: layers)
    return cfg, f"{args.workload} family at n={n}, batch {B}, depth {args.depth} (profiling case)"


# ---------------------------------------------------------------------------
# oracle timing (CPU, single thread, bounded sample of the same workload)
# ---------------------------------------------------------------------------

def oracle_sample_child(name: str, budget: float):
    """Times the oracle's own gate application (einsum) and inner product on
    sample 0 of the workload at full n, over gates spread evenly through the
    circuit, until `budget` seconds are spent; prints JSON."""
    import numpy as np
    from oracle import qsim_oracle as O
    cfg = W.WORKLOADS[name]
    n, layers = cfg["n"], cfg["layers"]()
    x, theta, g = W.draw_inputs(n, layers, 1, seed=0)
    gates = []
    for layer in layers:
        gates.extend(O.layer_gates(n, layer, x[0], theta))
    nparam = sum(len(d) for _, _, d in gates)
    psi = np.zeros(2 ** n, dtype=np.complex128)
    psi[0] = 1.0
    t = psi.reshape([2] * n)
    step = max(1, len(gates) // 64)
    order = list(range(0, len(gates), step))
    t_apply, cnt, t0 = 0.0, 0, time.perf_counter()
    i = 0
    while time.perf_counter() - t0 < budget and i < 10 * len(order):
        qubits, U, _ = gates[order[i % len(order)]]
        a = time.perf_counter()
        t = O.apply_local(t, U, qubits)
        t_apply += time.perf_counter() - a
        cnt += 1
        i += 1
    a = time.perf_counter()
    v = np.vdot(t.reshape(-1), t.reshape(-1))
    t_vdot = time.perf_counter() - a
    # adjoint_sample applies every gate 3 times (forward, psi and lambda
    # uncompute) plus one derivative application and one inner product per parameter
    n_apply = 3 * len(gates) + nparam
    per_eval = n_apply * (t_apply / cnt) + nparam * t_vdot
    print(json.dumps(dict(per_eval_s=per_eval, applies_timed=cnt, sample_s=time.perf_counter() - t0,
                          n_apply=n_apply, n_gates=len(gates), n_params=nparam, v=float(v.real))))


def oracle_baseline(name: str, budget: float):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", name,
                        "--oracle-budget", str(budget)], capture_output=True, text=True, env=env,
                       cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    B = W.WORKLOADS[name]["batch"]
    d["evals_per_s"] = 1.0 / d["per_eval_s"]
    d["sample"] = (f"1 sample of {name} at full n: {d['applies_timed']} of the oracle's gate "
                   f"applications (einsum, complex128) spread through the circuit plus one inner "
                   f"product, timed in {d['sample_s']:.1f} s on 1 thread and scaled to the "
                   f"{d['n_apply']} applications + {d['n_params']} inner products of one "
                   f"fwd+adjoint evaluation; batch {B} = {B} independent evaluations")
    return d


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def traffic_record(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None."""
    p = os.path.join(ROOT, "profiles", "traffic_per_launch.txt")
    if not os.path.exists(p):
        return None
    for line in open(p):
        f = line.split()
        if len(f) >= 3 and not line.startswith("#") and f[0] == kernel and f[1] == workload:
            return float(f[2])
    return None


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def gpu_arm(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2506_04891_gb300 import qlayer as Q

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    cfg, descr = workload_cfg(args)
    n, layers, B = cfg["n"], cfg["layers"](), cfg["batch"]
    circ = Q.Circuit(n, layers, dtype=cfg["dtype"])
    x_np, th_np, g_np = W.draw_inputs(n, layers, B, seed=rank)
    x = torch.tensor(x_np, device="cuda")
    th = torch.tensor(th_np, device="cuda")
    g = torch.tensor(g_np, device="cuda")
    psi = torch.empty((B, 1 << n), dtype=circ.state_dtype, device="cuda")
    ez = torch.empty((B, n), dtype=torch.float64, device="cuda")
    dth = torch.empty((circ.n_theta,), dtype=torch.float64, device="cuda")
    dx = torch.empty((B, circ.n_in), dtype=torch.float64, device="cuda")
    ws = circ.workspace(B)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    def step():
        Q.qc_forward(circ.handle, B, x.data_ptr(), th.data_ptr(), psi.data_ptr(), ez.data_ptr(),
                     ws.data_ptr(), ws.numel(), sh)
        Q.qc_backward(circ.handle, B, x.data_ptr(), th.data_ptr(), psi.data_ptr(), g.data_ptr(),
                      dth.data_ptr(), dx.data_ptr(), ws.data_ptr(), ws.numel(), sh)
        if world > 1:
            dist.all_reduce(dth)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    Q.qc_profile_enable(True)
    l0 = Q.qc_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = Q.qc_launch_count() - l0
    prof = Q.qc_profile_summary()
    Q.qc_profile_enable(False)
    ms = e0.elapsed_time(e1)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    ms_step = ms / args.steps

    # end to end through the C ABI from pinned host buffers
    xh = torch.tensor(x_np).pin_memory()
    thh = torch.tensor(th_np).pin_memory()
    gh = torch.tensor(g_np).pin_memory()
    ezh = torch.empty((B, n), dtype=torch.float64).pin_memory()
    dthh = torch.empty((circ.n_theta,), dtype=torch.float64).pin_memory()
    dxh = torch.empty((B, circ.n_in), dtype=torch.float64).pin_memory()
    stg = torch.empty(Q.qc_staging_bytes(circ.handle, B), dtype=torch.uint8, device="cuda")

    def e2e_step():
        Q.qc_step_host(circ.handle, B, xh.data_ptr(), thh.data_ptr(), gh.data_ptr(), ezh.data_ptr(),
                       dthh.data_ptr(), dxh.data_ptr(), psi.data_ptr(), ws.data_ptr(), ws.numel(),
                       stg.data_ptr(), sh)
    e2e_step()
    if world > 1:
        dist.barrier()
    a = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e2e_s = (time.perf_counter() - a) / args.steps
    te = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_s = float(te.item())
    h2d = xh.numel() * 8 + thh.numel() * 8 + gh.numel() * 8
    d2h = ezh.numel() * 8 + dthh.numel() * 8 + dxh.numel() * 8

    if rank == 0:
        peak, peak_src = measured_peaks()
        dom = max(prof.items(), key=lambda kv: kv[1][1]) if prof else None
        roof = None
        if dom:
            name, (cnt, tot_ms, by) = dom
            achieved = by / (tot_ms * 1e-3) / 1e9
            tr = traffic_record(name, args.workload)
            roof = {"bound": "hbm", "kernel": name, "launches": cnt, "avg_ms": tot_ms / cnt,
                    "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "peak_source": peak_src,
                    "traffic": tr,
                    "share_of_step": round(tot_ms / ms, 4)}
        per_kernel = {k: {"launches": v[0], "ms_per_step": round(v[1] / args.steps, 3),
                          "GBps": round(v[2] / max(v[1], 1e-9) * 1e-6, 1)} for k, v in prof.items()}
        # algorithmic floor of a step: one read + write of the batch state per
        # forward layer, <Z> one read, two states read + written per backward layer
        S = B * (1 << n) * (8 if cfg["dtype"] == "c64" else 16)
        L = len(layers)
        floor_bytes = 2 * S * L + S + 4 * S * L
        evals = world * B / (ms_step * 1e-3)
        out = {
            "metric": METRIC, "value": round(evals, 3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if cfg["dtype"] == "c64" else "f64", "data": "synthetic",
            "config": {"workload": descr, "n": n, "batch_per_gpu": B,
                       "global_batch": B * world, "layers": L, "n_theta": circ.n_theta,
                       "state_bytes": S, "l2": "inputs larger than L2: every pass streams the batch state",
                       "parallelism": f"dp{world}: batch sharded, d theta all-reduced" if world > 1 else "single GPU"},
            "amp_updates_per_s": round(world * B * (1 << n) * L / (ms_step * 1e-3), 1),
            "step_floor_frac": round(floor_bytes / (ms_step * 1e-3) / 1e9 / peak, 4),
            "roofline": roof,
            "kernels": per_kernel,
            "e2e": {"value": round(world * B / e2e_s, 3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk,
        }
        if world == 1 and not args.no_cpu_baseline and descr == DESCR[args.workload]:
            try:
                ob = oracle_baseline(args.workload, 15.0)
                out["cpu_baseline"] = {"value": round(ob["evals_per_s"], 6), "unit": UNIT,
                                       "cores": 1, "kind": "oracle", "sample": ob["sample"]}
            except Exception as e:  # report, do not hide
                out["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                       "sample": f"failed: {e}"}
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def reference_arm(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    times = []
    budget = 3.0
    for i in range(args.warmup + args.steps):
        d = oracle_baseline(args.workload, budget)
        if i >= args.warmup:
            times.append(d["per_eval_s"])
    per_eval = statistics.mean(times)
    val = 1.0 / per_eval
    B = W.WORKLOADS[args.workload]["batch"]
    out = {
        "metric": METRIC, "value": round(val, 6), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(per_eval * B * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": DESCR[args.workload], "batch_per_gpu": B},
        "cpu_baseline": {"value": round(val, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": d["sample"] + f"; each step re-times a {budget:.0f} s sample"},
        "e2e": {"value": round(val, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.oracle_sample:
        oracle_sample_child(args.oracle_sample, args.oracle_budget)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()

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
  python bench.py --impl reference ...   # the CPU oracle on every host core, bounded samples
  python bench.py --impl pergate ...     # complex128 per-gate torch path vs this library
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

L2_BYTES = 129 * 1024 * 1024  # GB300 L2
METRIC = "fwd+bwd circuit evals/s"
UNIT = "evals/s"
DESCR = {
    "zz26": "zz26: n=26, batch 8/GPU, complex64; RX(x) + 12x[RY, IsingZZ ring, CNOT ring]; fwd + <Z> + adjoint bwd",
    "hea4": "hea4: n=4, batch 8/GPU, complex128; RX(x) + 2x[RY, CNOT ring]; fwd + <Z> + adjoint bwd",
    "hea12": "hea12: n=12, batch 256/GPU, complex64; RX(x) + 10x[RZ, RY, RZ, CNOT ring]; fwd + <Z> + adjoint bwd",
    "hea12_c128": "hea12_c128: n=12, batch 256/GPU, complex128; RX(x) + 10x[RZ, RY, RZ, CNOT ring]; fwd + <Z> + adjoint bwd",
    "ibm20": "ibm20: n=20, batch 32/GPU, complex64; IBM native body depth 8; fwd + <Z> + adjoint bwd",
    "ionq20": "ionq20: n=20, batch 32/GPU, complex64; IonQ native body depth 8; fwd + <Z> + adjoint bwd",
    "serve20": "serve20: n=20, batch 2/GPU, complex64; RX(x) + 6x[RZ, RY, RZ, CNOT ring] (serving request circuit)",
    "serve24": "serve24: n=24, batch 2/GPU, complex64; RX(x) + 6x[RZ, RY, RZ, CNOT ring] (serving request circuit)",
}
# golden files of the oracle's values (tests/golden/<name>.npz, seed 0)
GOLDEN = {"hea4": "hea4", "hea12": "hea12", "hea12_c128": "hea12", "ibm20": "ibm20", "ionq20": "ionq20",
          "zz26": "zz26", "serve20": "serve20", "serve24": "serve24"}
# a full oracle fwd+adjoint evaluation takes under a few seconds: time whole
# evaluations; the others are extrapolated from timed gate applications
ORACLE_FULL = {"hea4", "hea12", "hea12_c128"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference", "pergate"])
    ap.add_argument("--workload", default="zz26", choices=sorted(DESCR))
    ap.add_argument("--oracle-worker", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-budget", type=float, default=12.0,
                    help="seconds of oracle work per baseline measurement (single and pool each)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=3,
                    help="steps of the separate per-kernel profiled pass after the timed region")
    # smaller cases of the same circuit family, for profiling captures
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--batch", type=int, default=None)
    ap.add_argument("--depth", type=int, default=None)
    return ap.parse_args()


def workload_cfg(args):
    cfg = dict(W.WORKLOADS[args.workload])
    if args.n is None and args.batch is None and args.depth is None:
        return cfg, DESCR[args.workload], True
    n = args.n or cfg["n"]
    B = args.batch or cfg["batch"]
    fam = {"zz26": lambda d: W.zz_circuit(n, d or 12), "hea12": lambda d: W.hea_circuit(n, d or 10),
           "hea12_c128": lambda d: W.hea_circuit(n, d or 10),
           "hea4": lambda d: W.hea_circuit(n, d or 2, block=("RY",)),
           "ibm20": lambda d: W.ibm_circuit(n, d or 8), "ionq20": lambda d: W.ionq_circuit(n, d or 8),
           "serve20": lambda d: W.hea_circuit(n, d or 6), "serve24": lambda d: W.hea_circuit(n, d or 6)}
    layers = fam[args.workload](args.depth)
    cfg.update(n=n, batch=B, layers=lambda: layers)
    return cfg, f"{args.workload} family at n={n}, batch {B}, depth {args.depth} (profiling case)", False


def host_cores():
    """(os.cpu_count(), lscpu's CPU count and model) of this host."""
    info = {"os_cpu_count": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() == "CPU(s)":
                info["lscpu_cpus"] = int(v.strip())
            elif k.strip() == "Model name":
                info["model"] = v.strip()
    except (OSError, ValueError, subprocess.TimeoutExpired):
        pass
    return info


# ---------------------------------------------------------------------------
# oracle timing (CPU): persistent single-thread workers
# ---------------------------------------------------------------------------

def oracle_worker(name: str, wid: int):
    """One single-threaded oracle worker.  Reads "run <seconds>" lines and
    answers each with one JSON line: how many fwd+adjoint evaluations of the
    workload its oracle work in that time amounts to.  Small workloads run
    whole evaluations (oracle.adjoint_sample on sample wid mod B, as it
    stands); the others time the oracle's own gate applications (einsum,
    complex128) on one full-size sample, continuing through the circuit from
    call to call, and scale to the applications and inner products one
    evaluation makes (extrapolated)."""
    import numpy as np
    from oracle import qsim_oracle as O
    cfg = W.WORKLOADS[name]
    n, layers, B = cfg["n"], cfg["layers"](), cfg["batch"]
    x, theta, g = W.draw_inputs(n, layers, B, seed=0)
    n_theta, n_in = O.num_params(n, layers)
    full = name in ORACLE_FULL
    if not full:
        gates = []
        for layer in layers:
            gates.extend(O.layer_gates(n, layer, x[wid % B], theta))
        nparam = sum(len(d) for _, _, d in gates)
        n_apply = 3 * len(gates) + nparam
        t = O.zero_state(n).reshape([2] * n)
        step = max(1, len(gates) // 64)
        order = list(range(0, len(gates), step))
        pos = 0
        a = time.perf_counter()
        v = np.vdot(t.reshape(-1), t.reshape(-1))
        t_vdot = time.perf_counter() - a
    print(json.dumps({"ready": True}), flush=True)
    for line in sys.stdin:
        cmd = line.split()
        if not cmd or cmd[0] != "run":
            break
        budget = float(cmd[1])
        t0 = time.perf_counter()
        if full:
            evals, b = 0, wid
            while True:
                O.adjoint_sample(n, layers, x[b % B], theta, g[b % B], n_theta, n_in)
                evals += 1
                b += 1
                if time.perf_counter() - t0 >= budget:
                    break
            sec = time.perf_counter() - t0
            print(json.dumps({"evals": evals, "seconds": sec, "extrapolated": False}), flush=True)
        else:
            cnt, t_apply = 0, 0.0
            while True:
                qubits, U, _ = gates[order[pos % len(order)]]
                a = time.perf_counter()
                t = O.apply_local(t, U, qubits)
                t_apply += time.perf_counter() - a
                cnt += 1
                pos += 1
                if time.perf_counter() - t0 >= budget:
                    break
            sec = time.perf_counter() - t0
            per_eval = n_apply * (t_apply / cnt) + nparam * t_vdot
            print(json.dumps({"evals": sec / per_eval, "seconds": sec, "extrapolated": True,
                              "applies": cnt, "n_apply": n_apply, "n_params": nparam}), flush=True)


class OraclePool:
    """`count` persistent oracle worker processes (fresh interpreters with one
    BLAS / OpenMP thread each), run concurrently."""

    def __init__(self, name: str, count: int):
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        self.procs = [subprocess.Popen([sys.executable, os.path.abspath(__file__), "--workload", name,
                                        "--oracle-worker", str(i)], stdin=subprocess.PIPE,
                                       stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env,
                                       cwd=ROOT) for i in range(count)]
        for p in self.procs:
            self._read(p)

    @staticmethod
    def _read(p):
        line = p.stdout.readline()
        if not line:
            raise RuntimeError("oracle worker failed: " + p.stderr.read()[-2000:])
        return json.loads(line)

    def run(self, budget: float):
        """All workers work `budget` seconds at once; returns (aggregate evals/s,
        wall seconds, per-worker records)."""
        a = time.perf_counter()
        for p in self.procs:
            p.stdin.write(f"run {budget}\n")
            p.stdin.flush()
        recs = [self._read(p) for p in self.procs]
        wall = time.perf_counter() - a
        return sum(r["evals"] / r["seconds"] for r in recs), wall, recs

    def close(self):
        for p in self.procs:
            try:
                p.stdin.write("quit\n")
                p.stdin.flush()
                p.wait(timeout=30)
            except Exception:
                p.kill()


def oracle_baseline(name: str, budget: float):
    """The oracle as it stands, timed on this host: one worker alone (1
    thread), then one worker per core at once (process pool)."""
    cores = host_cores()
    ncores = cores.get("os_cpu_count") or 1
    single = OraclePool(name, 1)
    try:
        s_rate, _, s_recs = single.run(budget)
    finally:
        single.close()
    pool = OraclePool(name, ncores)
    try:
        p_rate, p_wall, p_recs = pool.run(budget)
    finally:
        pool.close()
    extra = s_recs[0]["extrapolated"]
    how = ("whole oracle fwd+adjoint evaluations (oracle.adjoint_sample, complex128)" if not extra else
           f"the oracle's gate applications (einsum, complex128) on one full-size sample, "
           f"scaled to the {s_recs[0]['n_apply']} applications + {s_recs[0]['n_params']} inner products "
           f"of one fwd+adjoint evaluation (extrapolated)")
    sample = (f"{budget:.0f} s of {how}: 1 worker alone, then {ncores} workers at once "
              f"(one single-threaded process per core); value = the pool's aggregate rate")
    return {"value": round(p_rate, 6), "unit": UNIT, "cores": ncores, "kind": "oracle", "sample": sample,
            "single": round(s_rate, 6), "pool": round(p_rate, 6), "extrapolated": extra,
            "host": cores}


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
# modelled arithmetic of a step (for the complex128 compute roofline)
# ---------------------------------------------------------------------------

def flops_per_amp_fwd(n: int, layers) -> float:
    """Real floating-point operations per amplitude of one forward pass of
    the method (gate math only): a complex 2x2 gate on a pair costs 4 complex
    multiplies and 2 adds (14 flops per amplitude), a real one (RY) 6, a
    diagonal phase one complex multiply (6 per layer), a complex 4x4 brick gate
    30 per amplitude, permutations none.  The adjoint backward undoes every
    gate on psi and on lambda and forms the gradient inner products: about 2.5
    forward passes; one evaluation is modelled as 3.5 forward passes."""
    f = 0.0
    for kind, _s, _o, parity in layers:
        if kind in ("RX", "SX", "GPI2", "H"):
            f += 14 * n
        elif kind == "RY":
            f += 6 * n
        elif kind == "ROT":
            f += 6 * n + 12
        elif kind in ("RZ", "ISINGZZ_RING", "GPI", "Z", "S"):
            f += 6
        elif kind.endswith("_BRICK") and kind not in ("SWAP_BRICK",):
            f += 30 * ((n - parity) // 2)
    return f


def golden_errors(Q, circ, name, dtype):
    """Max |GPU - oracle| of every output on the golden samples of `name`
    (oracle values stored by tests/golden/make_goldens.py, seed-0 inputs):
    <Z>, d x, d theta summed over those samples, and psi at the stored
    indices.  Runs its own small forward + backward (outside the timing)."""
    import numpy as np
    import torch
    path = os.path.join(ROOT, "tests", "golden", GOLDEN.get(name, name) + ".npz")
    if not os.path.exists(path):
        return None
    G = np.load(path)
    cfg = W.WORKLOADS[name]
    n, layers = cfg["n"], cfg["layers"]()
    x, theta, g = W.draw_inputs(n, layers, cfg["batch"], seed=0)
    bs = [int(b) for b in G["samples"]]
    xt = torch.tensor(x[bs], device="cuda")
    tt = torch.tensor(theta, device="cuda")
    psi, ez = circ.forward(xt, tt, batch=len(bs))
    dth, dx = circ.backward(xt, tt, psi, torch.tensor(g[bs], device="cuda"))
    torch.cuda.synchronize()
    out = {"samples": len(bs)}
    out["ez"] = float(np.max(np.abs(ez.cpu().numpy() - G["ez"])))
    if circ.n_in:
        out["dx"] = float(np.max(np.abs(dx.cpu().numpy() - G["dx"])))
    if circ.n_theta:
        ref = G["dth_sum"] if "dth_sum" in G.files else G["dth"].sum(axis=0)
        out["dtheta_sum"] = float(np.max(np.abs(dth.cpu().numpy() - ref)))
    idx = torch.as_tensor(G["psi_idx"], device="cuda")
    got = torch.stack([psi[k][idx[k]] for k in range(len(bs))]).cpu().numpy().astype(np.complex128)
    out["psi"] = float(np.max(np.abs(got - G["psi_val"])))
    out["tolerance"] = ("complex128: 1e-12 relative" if dtype == "c128" else
                        "complex64: 2e-5 absolute (<Z>, d x; d theta 2e-5 x samples)")
    return out


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def gpu_arm(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2506_04891_gb300 import dist as D
    from paper_2506_04891_gb300 import qlayer as Q

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    cfg, descr, stock = workload_cfg(args)
    n, layers, B = cfg["n"], cfg["layers"](), cfg["batch"]
    circ = Q.Circuit(n, layers, dtype=cfg["dtype"])
    x_np, th_np, g_np = W.draw_inputs(n, layers, B, seed=rank)
    x = torch.tensor(x_np, device="cuda")
    th = torch.tensor(th_np, device="cuda")
    g = torch.tensor(g_np, device="cuda")
    psi = torch.empty((B, 1 << n), dtype=circ.state_dtype, device="cuda")
    ws = circ.workspace(B)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    def step():
        # this rank's shard: forward + <Z> + adjoint backward, then the d theta all-reduce
        return D.data_parallel_step(circ, x if circ.n_in else None, th if circ.n_theta else None, g,
                                    psi_out=psi, workspace=ws)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    l0 = Q.qc_launch_count()
    a0 = Q.qc_alloc_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = Q.qc_launch_count() - l0
    allocs = Q.qc_alloc_count() - a0
    ms = e0.elapsed_time(e1)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    ms_step = ms / args.steps

    # per-kernel split: a separate pass of the same steps with every launch
    # bracketed by CUDA events on its stream (the timed region above runs clean)
    psteps = max(1, min(args.profile_steps, args.steps))
    Q.qc_profile_enable(True)
    for _ in range(psteps):
        step()
    prof = Q.qc_profile_summary()
    Q.qc_profile_enable(False)

    # end to end through the C ABI from pinned host buffers
    xh = torch.tensor(x_np).pin_memory()
    thh = torch.tensor(th_np).pin_memory()
    gh = torch.tensor(g_np).pin_memory()
    ezh = torch.empty((B, n), dtype=torch.float64).pin_memory()
    dthh = torch.empty((max(circ.n_theta, 1),), dtype=torch.float64).pin_memory()
    dxh = torch.empty((B, max(circ.n_in, 1)), dtype=torch.float64).pin_memory()
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
    h2d = (xh.numel() if circ.n_in else 0) * 8 + (thh.numel() if circ.n_theta else 0) * 8 + gh.numel() * 8
    d2h = ezh.numel() * 8 + (dthh.numel() if circ.n_theta else 0) * 8 + (dxh.numel() if circ.n_in else 0) * 8

    if rank == 0:
        peak, peak_src = measured_peaks()
        peaks = {}
        for k, nm in ((0, "fp32_fmaf_tflops"), (1, "fp32x2_ffma2_tflops"), (2, "fp64_fma_tflops")):
            try:
                peaks[nm] = round(Q.qc_fma_peak(k), 2)
            except Exception as e:  # report, do not hide
                peaks[nm] = f"failed: {e}"
        dom = max(prof.items(), key=lambda kv: kv[1][1]) if prof else None
        roof = None
        if dom:
            name, (cnt, tot_ms, by) = dom
            achieved = by / (tot_ms * 1e-3) / 1e9
            tr = traffic_record(name, args.workload) if stock else None
            roof = {"bound": "hbm", "kernel": name, "launches": cnt // psteps, "avg_ms": tot_ms / cnt,
                    "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "peak_source": peak_src,
                    "traffic": tr, "share_of_step": round(tot_ms / psteps / ms_step, 4),
                    "timing": f"per-launch CUDA events on the launching stream over {psteps} profiled steps "
                              "after the timed region"}
        per_kernel = {k: {"launches": v[0] // psteps, "ms_per_step": round(v[1] / psteps, 3),
                          "GBps": round(v[2] / max(v[1], 1e-9) * 1e-6, 1)} for k, v in prof.items()}
        # algorithmic floor of a step: one read + write of the batch state per
        # forward layer, <Z> one read, two states read + written per backward layer
        w = 8 if cfg["dtype"] == "c64" else 16
        S = B * (1 << n) * w
        L = len(layers)
        floor_bytes = 2 * S * L + S + 4 * S * L
        evals = world * B / (ms_step * 1e-3)
        fl = 3.5 * flops_per_amp_fwd(n, layers) * B * (1 << n)
        compute = {"flops_per_step_model": fl, "achieved_tflops": round(fl / (ms_step * 1e-3) / 1e12, 3),
                   "peaks_measured": peaks}
        if cfg["dtype"] == "c128" and isinstance(peaks.get("fp64_fma_tflops"), float):
            t_fp64 = fl / (peaks["fp64_fma_tflops"] * 1e12)
            t_hbm = floor_bytes / (peak * 1e9)
            compute["fp64_floor_ms"] = round(t_fp64 * 1e3, 4)
            compute["hbm_floor_ms"] = round(t_hbm * 1e3, 4)
            compute["bound_of_min"] = "fp64" if t_fp64 > t_hbm else "hbm"
            compute["frac_of_min_roofline"] = round(max(t_fp64, t_hbm) / (ms_step * 1e-3), 4)
            if t_fp64 > t_hbm and roof is not None:
                # complex128 is bound by the FP64 pipe (1/64 of FP32 on this part):
                # the roofline is the step's modelled FP64 work against the measured
                # FP64 FMA peak
                roof = {"bound": "alu", "kernel": "whole step (modelled FP64 work)",
                        "achieved": round(fl / (ms_step * 1e-3) / 1e12, 4),
                        "peak": peaks["fp64_fma_tflops"], "unit": "TFLOP/s",
                        "frac": round(fl / (ms_step * 1e-3) / 1e12 / peaks["fp64_fma_tflops"], 4),
                        "peak_source": "measured (qc_fma_peak, FP64 FMA)", "traffic": None,
                        "dominant_kernel": dom[0], "share_of_step": round(dom[1][1] / psteps / ms_step, 4)}
        if roof is not None and roof.get("bound") == "hbm" and 2 * S <= L2_BYTES:
            # the carried states fit the 129 MB L2: the passes stream from L2, so
            # the algorithmic bytes per second are not an HBM figure
            roof["l2_resident"] = True
        out = {
            "metric": METRIC, "value": round(evals, 3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if cfg["dtype"] == "c64" else "f64", "data": "synthetic",
            "config": {"workload": descr, "n": n, "batch_per_gpu": B,
                       "global_batch": B * world, "layers": L, "n_theta": circ.n_theta,
                       "state_bytes": S,
                       "l2": ("inputs larger than L2: every pass streams the batch state" if S > 129e6 else
                              "state fits in L2 (launch / latency regime, no flush)"),
                       "parallelism": f"dp{world}: batch sharded, d theta all-reduced" if world > 1 else "single GPU"},
            "amp_updates_per_s": round(world * B * (1 << n) * L / (ms_step * 1e-3), 1),
            "step_floor_frac": round(floor_bytes / (ms_step * 1e-3) / 1e9 / peak, 4),
            "roofline": roof,
            "compute": compute,
            "kernels": per_kernel,
            "e2e": {"value": round(world * B / e2e_s, 3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "device_allocs_in_timed_region": allocs,
            "clocks": clk,
        }
        if stock:
            try:
                out["errors_vs_oracle"] = golden_errors(Q, circ, args.workload, cfg["dtype"])
            except Exception as e:  # report, do not hide
                out["errors_vs_oracle"] = f"failed: {e}"
        if world == 1 and not args.no_cpu_baseline and stock:
            try:
                out["cpu_baseline"] = oracle_baseline(args.workload, args.oracle_budget)
            except Exception as e:  # report, do not hide
                out["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle",
                                       "sample": f"failed: {e}"}
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def reference_arm(args):
    """The oracle, as it stands, on this host's cores: every step is a bounded
    sample (`budget` seconds of oracle work on every core at once); the value
    is the aggregate evaluation rate of all cores."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    budget = 3.0
    cores = host_cores()
    ncores = cores.get("os_cpu_count") or 1
    pool = OraclePool(args.workload, ncores)
    rates, walls = [], []
    try:
        for i in range(args.warmup + args.steps):
            rate, wall, recs = pool.run(budget)
            if i >= args.warmup:
                rates.append(rate)
                walls.append(wall)
    finally:
        pool.close()
    val = statistics.mean(rates)
    extra = recs[0]["extrapolated"]
    B = W.WORKLOADS[args.workload]["batch"]
    sample = (f"each step: {budget:.0f} s of oracle work in {ncores} single-threaded processes at once "
              + ("(whole fwd+adjoint evaluations)" if not extra else
                 "(the oracle's gate applications on one full-size sample each, scaled to one "
                 "fwd+adjoint evaluation: extrapolated)"))
    out = {
        "metric": METRIC, "value": round(val, 6), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(statistics.mean(walls) * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": DESCR[args.workload], "batch_per_gpu": B,
                   "step": "a bounded sample of the workload (see cpu_baseline.sample)"},
        "cpu_baseline": {"value": round(val, 6), "unit": UNIT, "cores": ncores, "kind": "oracle",
                         "sample": sample, "extrapolated": extra, "host": cores},
        "e2e": {"value": round(val, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def pergate_arm(args):
    """The plain complex128 per-gate PyTorch path (torch.einsum per gate,
    autograd backward; pergate_torch.py) and this library on the same GPU and
    the same inputs: both timed with CUDA events, the speedup of the library's
    chosen form over the per-gate path, and the library's largest difference
    from the per-gate results (which match the oracle to 1e-12)."""
    import numpy as np
    import torch

    import pergate_torch as PG
    from paper_2506_04891_gb300 import qlayer as Q

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    cfg, descr, _ = workload_cfg(args)
    n, layers, B = cfg["n"], cfg["layers"](), cfg["batch"]
    free, _ = torch.cuda.mem_get_info()
    budget = int(free * 0.85)
    fit = PG.max_batch(n, layers, budget, B)
    note = None
    if fit == 0:
        # the per-gate path keeps every gate's input for autograd: take the
        # largest n of the same family at which the batch fits
        while n > 2 and PG.max_batch(n, layers, budget, B) < B:
            n -= 1
            args.n, args.depth = n, None
            cfg, descr, _ = workload_cfg(args)
            layers = cfg["layers"]()
        fit = PG.max_batch(n, layers, budget, B)
        note = f"the stated n does not fit the per-gate path's autograd memory; largest fitting n = {n}"
    elif fit < B:
        note = f"batch {B} does not fit the per-gate path's autograd memory; largest fitting batch = {fit}"
    Bp = fit
    x_np, th_np, g_np = W.draw_inputs(n, layers, Bp, seed=0)
    x = torch.tensor(x_np, device="cuda")
    th = torch.tensor(th_np, device="cuda")
    g = torch.tensor(g_np, device="cuda")
    xin = x if x.numel() else None

    def time_it(fn):
        for _ in range(args.warmup):
            r = fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps, r

    ms_pg, r_pg = time_it(lambda: PG.fwd_bwd(n, layers, xin, th, g))
    peak_mem = torch.cuda.max_memory_allocated()
    torch.cuda.empty_cache()
    circ = Q.Circuit(n, layers, dtype=cfg["dtype"])
    psi = torch.empty((Bp, 1 << n), dtype=circ.state_dtype, device="cuda")
    ws = circ.workspace(Bp)

    def ours():
        _, ez = circ.forward(xin, th if circ.n_theta else None, batch=Bp, psi_out=psi, workspace=ws)
        dth, dx = circ.backward(xin, th if circ.n_theta else None, psi, g, workspace=ws)
        return ez, dth, dx
    ms_us, r_us = time_it(ours)
    err = {"ez": float((r_us[0] - r_pg[0]).abs().max())}
    if r_pg[1] is not None:
        err["dtheta_sum"] = float((r_us[1] - r_pg[1]).abs().max())
        err["dtheta_tolerance"] = 2e-5 * Bp if cfg["dtype"] == "c64" else "1e-12 relative"
    if r_pg[2] is not None:
        err["dx"] = float((r_us[2][:, :r_pg[2].shape[1]] - r_pg[2]).abs().max())
    out = {
        "metric": METRIC, "value": round(Bp / (ms_pg * 1e-3), 3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_pg, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "pergate",
        "config": {"workload": descr, "n": n, "batch_per_gpu": Bp, "note": note,
                   "pergate": "torch.einsum per gate, complex128, torch.autograd backward",
                   "pergate_peak_bytes": peak_mem, "gates": PG.gate_count(n, layers)},
        "library": {"dtype": cfg["dtype"], "ms_per_step": round(ms_us, 3),
                    "value": round(Bp / (ms_us * 1e-3), 3)},
        "speedup_fwd_bwd": round(ms_pg / ms_us, 2),
        "library_minus_pergate_max_abs": err,
    }
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.oracle_worker is not None:
        oracle_worker(args.workload, int(args.oracle_worker))
        return
    if args.impl == "reference":
        reference_arm(args)
    elif args.impl == "pergate":
        pergate_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()

"""Continuous batching of circuit requests on one GPU.

A request is one forward + <Z> + adjoint-gradient evaluation of the serving
circuit (RX(x) embedding, 6 x [RZ, RY, RZ, CNOT ring]) for its own qubit count
n and batch B.  Requests arrive over time; the server admits a request (or a
chunk of its batch) as soon as a stream slot is free and its device footprint
fits in the HBM budget next to the work already in flight, so requests that
arrive while others run overlap with them on the device.  A request whose
footprint alone exceeds the budget is split along the batch; its chunks' d theta
are summed.

The host side (admission, chunking, bookkeeping) lives in ``Scheduler`` and runs
without a GPU; ``GpuExecutor`` issues the asynchronous copies and C-ABI calls on
CUDA streams and polls events (the host never blocks on one request).
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np

from . import workloads as W


@dataclasses.dataclass(eq=False)
class Request:
    rid: int
    n: int
    batch: int
    x: np.ndarray       # [B, n] float64
    theta: np.ndarray   # [P] float64
    g: np.ndarray       # [B, n] upstream d loss / d <Z>
    arrival: float = 0.0


@dataclasses.dataclass(eq=False)
class Result:
    rid: int
    ez: np.ndarray
    dtheta: np.ndarray
    dx: np.ndarray
    arrival: float
    admitted: float = math.nan
    done: float = math.nan
    chunks: int = 0

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def make_requests(count: int, seed: int = 0, n_range=(8, 24), b_range=(1, 512)):
    """Seeded serving stream (shapes only; arrival times are set by the caller)."""
    out = []
    for rid, (n, b) in enumerate(W.serving_requests(count, seed, n_range, b_range)):
        layers = W.serving_circuit(n)
        x, theta, g = W.draw_inputs(n, layers, b, seed=seed * 100003 + rid)
        out.append(Request(rid, n, b, x, theta, g))
    return out


class Scheduler:
    """Admission by device footprint; no GPU needed.

    footprint(n, b) -> bytes a chunk of b samples of an n-qubit request holds on
    the device while it runs.  ``slots`` bounds the chunks in flight.
    """

    def __init__(self, budget_bytes: int, slots: int, footprint):
        self.budget = int(budget_bytes)
        self.slots = int(slots)
        self.footprint = footprint
        self.in_flight = {}   # chunk key -> bytes
        self.used = 0

    def max_chunk(self, n: int, batch: int) -> int:
        """Largest b <= batch whose footprint fits in the whole budget (0 if none)."""
        lo, hi = 0, batch
        while lo < hi:
            mid = (lo + hi + 1) // 2
            if self.footprint(n, mid) <= self.budget:
                lo = mid
            else:
                hi = mid - 1
        return lo

    def split(self, req: Request):
        """Batch ranges of the request's chunks."""
        m = self.max_chunk(req.n, req.batch)
        if m == 0:
            raise ValueError(f"request {req.rid}: one sample of n={req.n} exceeds the HBM budget")
        return [(lo, min(lo + m, req.batch)) for lo in range(0, req.batch, m)]

    def can_admit(self, n: int, b: int) -> bool:
        return len(self.in_flight) < self.slots and self.used + self.footprint(n, b) <= self.budget

    def admit(self, key, n: int, b: int):
        fp = self.footprint(n, b)
        self.in_flight[key] = fp
        self.used += fp

    def release(self, key):
        self.used -= self.in_flight.pop(key)


class GpuExecutor:
    """Runs chunks on CUDA streams through the C ABI (asynchronous)."""

    def __init__(self, slots: int, dtype: str = "c64", ckpt_every: int = 0):
        import torch
        from . import qlayer as Q
        self.torch = torch
        self.Q = Q
        self.dtype = dtype
        self.ckpt = ckpt_every
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.free_streams = list(range(slots))
        self.circuits = {}

    def circuit(self, n: int):
        c = self.circuits.get(n)
        if c is None:
            c = self.Q.Circuit(n, W.serving_circuit(n), dtype=self.dtype, ckpt_every=self.ckpt)
            self.circuits[n] = c
        return c

    def footprint(self, n: int, b: int) -> int:
        c = self.circuit(n)
        w = 8 if self.dtype == "c64" else 16
        return (b << n) * w + c.workspace_bytes(b) + 16 * b * (3 * n + 2) + 8 * c.n_theta * 2

    def launch(self, req: Request, lo: int, hi: int):
        torch, Q = self.torch, self.Q
        si = self.free_streams.pop()
        st = self.streams[si]
        c = self.circuit(req.n)
        b = hi - lo
        with torch.cuda.stream(st):
            xh = torch.from_numpy(np.ascontiguousarray(req.x[lo:hi])).pin_memory()
            th = torch.from_numpy(np.ascontiguousarray(req.theta)).pin_memory()
            gh = torch.from_numpy(np.ascontiguousarray(req.g[lo:hi])).pin_memory()
            x = xh.to("cuda", non_blocking=True)
            t = th.to("cuda", non_blocking=True)
            g = gh.to("cuda", non_blocking=True)
            psi = torch.empty((b, 1 << req.n), dtype=c.state_dtype, device="cuda")
            ez = torch.empty((b, req.n), dtype=torch.float64, device="cuda")
            dth = torch.empty((c.n_theta,), dtype=torch.float64, device="cuda")
            dx = torch.empty((b, c.n_in), dtype=torch.float64, device="cuda")
            ws = torch.empty(max(c.workspace_bytes(b), 256), dtype=torch.uint8, device="cuda")
            h = st.cuda_stream
            Q.qc_forward(c.handle, b, x.data_ptr(), t.data_ptr(), psi.data_ptr(), ez.data_ptr(),
                         ws.data_ptr(), ws.numel(), h)
            Q.qc_backward(c.handle, b, x.data_ptr(), t.data_ptr(), psi.data_ptr(), g.data_ptr(),
                          dth.data_ptr(), dx.data_ptr(), ws.data_ptr(), ws.numel(), h)
            out = (torch.empty(ez.shape, dtype=torch.float64).pin_memory(),
                   torch.empty(dth.shape, dtype=torch.float64).pin_memory(),
                   torch.empty(dx.shape, dtype=torch.float64).pin_memory())
            out[0].copy_(ez, non_blocking=True)
            out[1].copy_(dth, non_blocking=True)
            out[2].copy_(dx, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        # keep device buffers alive until the event completes
        return dict(stream=si, event=ev, keep=(x, t, g, psi, ez, dth, dx, ws, xh, th, gh), out=out)

    def done(self, handle) -> bool:
        return handle["event"].query()

    def finish(self, handle):
        self.free_streams.append(handle["stream"])
        ez, dth, dx = (a.numpy().copy() for a in handle["out"])
        handle.clear()
        return ez, dth, dx


class Server:
    """Continuous batching loop over a request stream."""

    def __init__(self, executor, scheduler: Scheduler):
        self.ex = executor
        self.sch = scheduler

    def run(self, requests, arrivals=None, clock=time.perf_counter):
        """Serves `requests` (arriving at `arrivals` seconds after the start, or
        all at once); returns {rid: Result} and stats."""
        reqs = list(requests)
        if arrivals is None:
            arrivals = [0.0] * len(reqs)
        order = sorted(range(len(reqs)), key=lambda i: arrivals[i])
        t0 = clock()
        pending = []               # [req, [(lo, hi), ...]] in arrival order
        results = {}
        partial = {}
        running = []
        nxt = 0
        total = len(reqs)
        while len(results) < total:
            now = clock() - t0
            while nxt < len(order) and arrivals[order[nxt]] <= now:
                r = reqs[order[nxt]]
                r.arrival = arrivals[order[nxt]]
                pending.append([r, self.sch.split(r)])
                results_entry = Result(r.rid, np.zeros((r.batch, r.n)), np.zeros(len(r.theta)),
                                       np.zeros((r.batch, r.x.shape[1])), r.arrival)
                partial[r.rid] = [results_entry, 0, len(pending[-1][1]), {}]
                nxt += 1
            # completions
            still = []
            for key, req, lo, hi, h in running:
                if self.ex.done(h):
                    ez, dth, dx = self.ex.finish(h)
                    self.sch.release(key)
                    ent = partial[req.rid]
                    res = ent[0]
                    res.ez[lo:hi] = ez
                    res.dx[lo:hi] = dx
                    ent[3][lo] = dth
                    res.chunks += 1
                    ent[1] += 1
                    if ent[1] == ent[2]:
                        for k in sorted(ent[3]):  # fixed order: batch position
                            res.dtheta += ent[3][k]
                        res.done = clock() - t0
                        results[req.rid] = res
                        del partial[req.rid]
                else:
                    still.append((key, req, lo, hi, h))
            running = still
            # admissions: first fit in arrival order
            for item in pending:
                req, chunks = item
                while chunks and self.sch.can_admit(req.n, chunks[0][1] - chunks[0][0]):
                    lo, hi = chunks.pop(0)
                    key = (req.rid, lo)
                    self.sch.admit(key, req.n, hi - lo)
                    ent = partial[req.rid][0]
                    if math.isnan(ent.admitted):
                        ent.admitted = clock() - t0
                    running.append((key, req, lo, hi, self.ex.launch(req, lo, hi)))
            pending = [item for item in pending if item[1]]
            if not running and not pending and nxt < len(order):
                time.sleep(max(0.0, min(0.001, arrivals[order[nxt]] - (clock() - t0))))
        wall = clock() - t0
        lat = np.array([r.latency for r in results.values()])
        stats = dict(requests=total, wall_s=wall, req_per_s=total / wall,
                     evals_per_s=sum(r.batch for r in reqs) / wall,
                     p50_ms=float(np.percentile(lat, 50) * 1e3), p99_ms=float(np.percentile(lat, 99) * 1e3))
        return results, stats


def poisson_arrivals(count: int, rate: float, seed: int = 0):
    rng = np.random.default_rng(seed + 17)
    return np.cumsum(rng.exponential(1.0 / rate, size=count)).tolist()


def serve_benchmark(count: int = 10000, slots: int = 4, budget_frac: float = 0.8, seed: int = 0,
                    n_range=(8, 24), b_range=(1, 512)):
    """Closed-loop throughput, then a Poisson stream at 0.8 x that rate; returns stats."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    ex = GpuExecutor(slots)
    sch = Scheduler(int(free * budget_frac), slots, ex.footprint)
    reqs = make_requests(count, seed, n_range, b_range)
    # warm up the kernels and plans of every qubit count
    Server(ex, Scheduler(int(free * budget_frac), slots, ex.footprint)).run(
        [r for r in make_requests(24, seed + 1, n_range, (1, 4))])
    _, closed = Server(ex, sch).run(reqs)
    rate = 0.8 * closed["req_per_s"]
    reqs = make_requests(count, seed, n_range, b_range)
    _, opened = Server(ex, Scheduler(int(free * budget_frac), slots, ex.footprint)).run(
        reqs, poisson_arrivals(count, rate, seed))
    return dict(closed_loop=closed, poisson=opened, arrival_rate=rate, slots=slots)


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=10000)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--nmax", type=int, default=24)
    ap.add_argument("--bmax", type=int, default=512)
    a = ap.parse_args()
    print(json.dumps(serve_benchmark(a.requests, a.slots, n_range=(8, a.nmax), b_range=(1, a.bmax))))

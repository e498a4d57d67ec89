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


ALIGN = 256  # every chunk's region in the device arena starts on a 256-byte boundary


def _align(v: int) -> int:
    return (v + ALIGN - 1) // ALIGN * ALIGN


class Scheduler:
    """Admission by device footprint; no GPU needed.

    footprint(n, b) -> bytes a chunk of b samples of an n-qubit request holds on
    the device while it runs.  The device memory is one arena of budget_bytes:
    admitting a chunk reserves a contiguous region of it (first fit), which
    the executor carves the chunk's buffers from, and releasing it frees the
    region, so no chunk allocates device memory.  ``slots`` bounds the chunks
    in flight.
    """

    def __init__(self, budget_bytes: int, slots: int, footprint):
        self.budget = int(budget_bytes) // ALIGN * ALIGN
        self.slots = int(slots)
        self.footprint = footprint
        self.in_flight = {}   # chunk key -> (offset, bytes)
        self.used = 0
        self.free = [(0, self.budget)]  # sorted, disjoint (offset, bytes) gaps

    def max_chunk(self, n: int, batch: int) -> int:
        """Largest b <= batch whose footprint fits in the whole budget (0 if none)."""
        lo, hi = 0, batch
        while lo < hi:
            mid = (lo + hi + 1) // 2
            if _align(self.footprint(n, mid)) <= self.budget:
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

    def _gap(self, need: int):
        for i, (off, size) in enumerate(self.free):
            if size >= need:
                return i
        return -1

    def can_admit(self, n: int, b: int) -> bool:
        return len(self.in_flight) < self.slots and self._gap(_align(self.footprint(n, b))) >= 0

    def admit(self, key, n: int, b: int) -> int:
        """Reserves the chunk's region; returns its byte offset in the arena."""
        need = _align(self.footprint(n, b))
        i = self._gap(need)
        if i < 0:
            raise RuntimeError("admit without room (check can_admit first)")
        off, size = self.free[i]
        if size == need:
            self.free.pop(i)
        else:
            self.free[i] = (off + need, size - need)
        self.in_flight[key] = (off, need)
        self.used += need
        return off

    def release(self, key):
        off, need = self.in_flight.pop(key)
        self.used -= need
        self.free.append((off, need))
        self.free.sort()
        merged = []
        for o, sz in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + sz)
            else:
                merged.append((o, sz))
        self.free = merged


class GpuExecutor:
    """Runs chunks on CUDA streams through the C ABI (asynchronous).

    All device memory of the chunks in flight is one arena, bound once to the
    scheduler's budget (``bind``); a chunk's buffers (state, workspace, inputs
    and outputs) are carved from the region the scheduler reserved for it.
    Every stream slot has pinned host staging buffers, allocated once for
    requests up to ``max_n`` qubits and ``max_b`` samples per chunk.  So
    serving a request allocates neither device nor pinned memory, and the
    compute calls themselves allocate nothing.
    """

    def __init__(self, slots: int, dtype: str = "c64", ckpt_every: int = 0, max_n: int = 24,
                 max_b: int = 512):
        import torch
        from . import qlayer as Q
        self.torch = torch
        self.Q = Q
        self.dtype = dtype
        self.ckpt = ckpt_every
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.free_streams = list(range(slots))
        self.circuits = {}
        self._layouts = {}
        self.arena = None
        nt = W.circuit_params(max_n, W.serving_circuit(max_n))[0]
        big = max_b * max_n

        def pin(k):
            return torch.empty(k, dtype=torch.float64).pin_memory()
        self.pinned = [dict(x=pin(big), theta=pin(nt), g=pin(big), ez=pin(big), dth=pin(nt), dx=pin(big))
                       for _ in range(slots)]
        self.max_n, self.max_b = max_n, max_b

    def bind(self, budget_bytes: int):
        """Allocates (or keeps, if large enough) the device arena."""
        if self.arena is None or self.arena.numel() < budget_bytes:
            self.arena = None
            self.arena = self.torch.empty(int(budget_bytes), dtype=self.torch.uint8, device="cuda")

    def circuit(self, n: int):
        c = self.circuits.get(n)
        if c is None:
            c = self.Q.Circuit(n, W.serving_circuit(n), dtype=self.dtype, ckpt_every=self.ckpt)
            self.circuits[n] = c
        return c

    def layout(self, n: int, b: int):
        """Byte offsets of a chunk's buffers inside its region, and its size
        (memoised: admission asks for it on every pass of the serving loop)."""
        key = (n, b)
        hit = self._layouts.get(key)
        if hit is not None:
            return hit
        hit = self._layout(n, b)
        self._layouts[key] = hit
        return hit

    def _layout(self, n: int, b: int):
        c = self.circuit(n)
        w = 8 if self.dtype == "c64" else 16
        sizes = [("ws", max(c.workspace_bytes(b), 256)), ("psi", (b << n) * w),
                 ("x", 8 * b * max(c.n_in, 1)), ("theta", 8 * max(c.n_theta, 1)), ("g", 8 * b * n),
                 ("ez", 8 * b * n), ("dth", 8 * max(c.n_theta, 1)), ("dx", 8 * b * max(c.n_in, 1))]
        off, out = 0, {}
        for name, nb in sizes:
            out[name] = (off, nb)
            off = _align(off + nb)
        return out, off

    def footprint(self, n: int, b: int) -> int:
        return self.layout(n, b)[1]

    def launch(self, req: Request, lo: int, hi: int, offset: int = 0):
        torch, Q = self.torch, self.Q
        if req.n > self.max_n or hi - lo > self.max_b:
            raise ValueError(f"request {req.rid}: beyond the executor's staging sizes")
        si = self.free_streams.pop()
        st = self.streams[si]
        pin = self.pinned[si]
        c = self.circuit(req.n)
        b, n = hi - lo, req.n
        lay, _ = self.layout(n, b)
        base = self.arena.data_ptr() + offset

        def dev(name, count):
            o = offset + lay[name][0]
            return self.arena[o: o + 8 * count].view(torch.float64)
        nx, nt, ng = b * c.n_in, c.n_theta, b * n
        pin["x"][:nx].numpy()[:] = req.x[lo:hi].reshape(-1)
        pin["theta"][:nt].numpy()[:] = req.theta
        pin["g"][:ng].numpy()[:] = req.g[lo:hi].reshape(-1)
        with torch.cuda.stream(st):
            dev("x", nx).copy_(pin["x"][:nx], non_blocking=True)
            dev("theta", nt).copy_(pin["theta"][:nt], non_blocking=True)
            dev("g", ng).copy_(pin["g"][:ng], non_blocking=True)
            p = {k: base + v[0] for k, v in lay.items()}
            h = st.cuda_stream
            Q.qc_forward(c.handle, b, p["x"], p["theta"], p["psi"], p["ez"], p["ws"], lay["ws"][1], h)
            Q.qc_backward(c.handle, b, p["x"], p["theta"], p["psi"], p["g"], p["dth"], p["dx"], p["ws"],
                          lay["ws"][1], h)
            pin["ez"][:ng].copy_(dev("ez", ng), non_blocking=True)
            pin["dth"][:nt].copy_(dev("dth", nt), non_blocking=True)
            pin["dx"][:nx].copy_(dev("dx", nx), non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        return dict(stream=si, event=ev, shape=(b, n, nt, c.n_in))

    def done(self, handle) -> bool:
        return handle["event"].query()

    def finish(self, handle):
        b, n, nt, nin = handle["shape"]
        pin = self.pinned[handle["stream"]]
        ez = pin["ez"][: b * n].numpy().reshape(b, n).copy()
        dth = pin["dth"][:nt].numpy().copy()
        dx = pin["dx"][: b * nin].numpy().reshape(b, nin).copy()
        self.free_streams.append(handle["stream"])
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
        bind = getattr(self.ex, "bind", None)
        if bind is not None:
            bind(self.sch.budget)
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
                    off = self.sch.admit(key, req.n, hi - lo)
                    ent = partial[req.rid][0]
                    if math.isnan(ent.admitted):
                        ent.admitted = clock() - t0
                    running.append((key, req, lo, hi, self.ex.launch(req, lo, hi, off)))
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
                    n_range=(8, 24), b_range=(1, 512), closed_sample: int = 1000):
    """The serving workload: a seeded stream of `count` requests (n and B
    uniform in the ranges).  The closed-loop throughput is measured on the
    stream's first `closed_sample` requests (all queued at once); the whole
    stream then arrives as a Poisson process at 0.8 x that rate.  Returns the
    statistics of both runs."""
    import torch
    from . import qlayer as Q
    free, _ = torch.cuda.mem_get_info()
    ex = GpuExecutor(slots, max_n=n_range[1], max_b=b_range[1])
    budget = int(free * budget_frac)

    def sched():
        return Scheduler(budget, slots, ex.footprint)
    # warm up: every qubit count's circuit (qc_create allocates its <Z>
    # scratch) and one small request of each, before anything is measured
    warm = []
    for k, n in enumerate(range(n_range[0], n_range[1] + 1)):
        ex.circuit(n)
        r = make_requests(1, seed + 1 + k, (n, n), (1, 2))[0]
        r.rid = k
        warm.append(r)
    Server(ex, sched()).run(warm)
    torch.cuda.synchronize()
    reqs = make_requests(count, seed, n_range, b_range)
    sample = reqs[: min(closed_sample, count)]
    a0 = Q.qc_alloc_count()
    _, closed = Server(ex, sched()).run(sample)
    rate = 0.8 * closed["req_per_s"]
    reqs = make_requests(count, seed, n_range, b_range)
    res, opened = Server(ex, sched()).run(reqs, poisson_arrivals(count, rate, seed))
    allocs = Q.qc_alloc_count() - a0
    lat = np.array([r.latency for r in res.values()])
    wait = np.array([r.admitted - r.arrival for r in res.values()])
    opened.update(p90_ms=float(np.percentile(lat, 90) * 1e3), mean_ms=float(lat.mean() * 1e3),
                  admit_wait_p50_ms=float(np.percentile(wait, 50) * 1e3),
                  admit_wait_p99_ms=float(np.percentile(wait, 99) * 1e3),
                  split_requests=int(sum(r.chunks > 1 for r in res.values())),
                  chunks=int(sum(r.chunks for r in res.values())))
    return dict(closed_loop=closed, closed_loop_requests=len(sample), poisson=opened, arrival_rate=rate,
                slots=slots, budget_bytes=budget, n_range=list(n_range), b_range=list(b_range),
                library_device_allocs_during_runs=allocs,
                request_evals=int(sum(r.batch for r in reqs)))


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=10000)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--nmax", type=int, default=24)
    ap.add_argument("--bmax", type=int, default=512)
    ap.add_argument("--closed-sample", type=int, default=1000)
    a = ap.parse_args()
    print(json.dumps(serve_benchmark(a.requests, a.slots, n_range=(8, a.nmax), b_range=(1, a.bmax),
                                     closed_sample=a.closed_sample)))

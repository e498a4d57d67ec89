"""World-size-2 gloo tests of the batch-sharded data-parallel step (CPU).

Each rank runs paper_2506_04891_gb300.dist.data_parallel_step on its shard
with a CPU stand-in circuit (the oracle stands in for the GPU kernels, which
these CPU ranks cannot run; it has the forward / backward signature of
qlayer.Circuit), so the step function itself and its d theta all-reduce are
exercised; the parent checks every rank against the full-batch oracle.  A second test makes one rank fail on the host
and checks that the other sees an error instead of hanging.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2506_04891_gb300 import dist as D
from paper_2506_04891_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


class _OracleCircuit:
    """CPU stand-in with qlayer.Circuit's forward / backward signature."""

    def __init__(self, n, layers):
        self.n, self.layers = n, layers
        self.calls = []

    def forward(self, x, theta, batch=None, psi_out=None, workspace=None):
        from oracle import qsim_oracle as O
        self.calls.append(("forward", psi_out is not None, workspace is not None))
        psi = O.forward(self.n, self.layers, x.numpy(), theta.numpy())
        ez = O.expect_z(psi, self.n)
        return torch.tensor(psi), torch.tensor(ez)

    def backward(self, x, theta, psi_out, g, workspace=None):
        from oracle import qsim_oracle as O
        self.calls.append(("backward", workspace is not None))
        _, dth, _, dx = O.adjoint(self.n, self.layers, x.numpy(), theta.numpy(), g.numpy())
        return torch.tensor(dth), torch.tensor(dx)


def _worker(rank, world, port, out_q, mode):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import datetime
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    try:
        from oracle import qsim_oracle as O
        n, B = 5, 5
        layers = W.zz_circuit(n, 2)
        x, theta, g = W.draw_inputs(n, layers, B, seed=0)
        lo, hi = D.shard_bounds(B, world, rank)
        if mode == "fail" and rank == 1:
            raise RuntimeError("planted host-side failure on rank 1")
        circ = _OracleCircuit(n, layers)
        ez, t, dx = D.data_parallel_step(circ, torch.tensor(x[lo:hi]), torch.tensor(theta),
                                         torch.tensor(g[lo:hi]), workspace="ws")
        assert circ.calls == [("forward", False, True), ("backward", True)]
        out_q.put((rank, lo, hi, ez.numpy(), t.numpy(), dx.numpy()))
    except Exception as e:  # reported to the parent
        out_q.put((rank, "error", repr(e)))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _run(mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q, mode)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
    return res


def test_shard_bounds_cover_batch():
    for B in (1, 5, 8, 31):
        for world in (1, 2, 3, 8):
            spans = [D.shard_bounds(B, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == B
            for (a, b), (c, d) in zip(spans, spans[1:]):
                assert b == c and b >= a
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1


def test_gloo_two_ranks_match_full_batch():
    from oracle import qsim_oracle as O
    res = _run("ok")
    assert all(r[1] != "error" for r in res), res
    n, B = 5, 5
    layers = W.zz_circuit(n, 2)
    x, theta, g = W.draw_inputs(n, layers, B, seed=0)
    ez, dth, _, dx = O.adjoint(n, layers, x, theta, g)
    for rank, lo, hi, ez_r, dth_r, dx_r in res:
        assert np.allclose(dth_r, dth, atol=1e-12)
        assert np.allclose(ez_r, ez[lo:hi], atol=1e-12)
        assert np.allclose(dx_r, dx[lo:hi], atol=1e-12)


def test_gloo_rank_failure_is_reported_not_hung():
    res = _run("fail")
    by_rank = {r[0]: r for r in res}
    assert by_rank[1][1] == "error"
    # rank 0 reaches the collective alone: it must end with an error (timeout
    # or peer closed), not hang
    assert by_rank[0][1] == "error", by_rank[0]

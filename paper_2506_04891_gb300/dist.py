"""Data parallelism over the input batch (one process per GPU).

Every sample's state evolves independently (Sec. 3: batching over input
data), so the batch shards across ranks with no exchange on the data path.
The one real exchange is the gradient of the shared trainable angles: each
rank's d theta is a sum over its shard, and the batch total is their sum
(one all-reduce of n_theta float64 values).  d x and <Z> stay sharded.
"""
from __future__ import annotations


def shard_bounds(global_batch: int, world: int, rank: int):
    """Contiguous shard [lo, hi) of `rank`; sizes differ by at most one."""
    if world <= 0 or not (0 <= rank < world):
        raise ValueError("bad world/rank")
    base, extra = divmod(global_batch, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi


def allreduce_dtheta(dtheta, group=None):
    """Sums d theta over ranks in place (float64 tensor on the rank's device)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(dtheta, op=dist.ReduceOp.SUM, group=group)
    return dtheta


def data_parallel_step(circuit, x_shard, theta, g_shard, group=None, psi_out=None, workspace=None):
    """Forward + <Z> + adjoint backward of this rank's shard, then the d theta
    all-reduce.  `circuit` is a ``qlayer.Circuit`` (or anything with its
    forward / backward signature); psi_out and workspace, if given, are reused
    across steps.  Returns (ez_shard, dtheta_total, dx_shard)."""
    psi, ez = circuit.forward(x_shard, theta, batch=g_shard.shape[0], psi_out=psi_out, workspace=workspace)
    dth, dx = circuit.backward(x_shard, theta, psi, g_shard, workspace=workspace)
    allreduce_dtheta(dth, group)
    return ez, dth, dx

"""Sharding of random initial states over ranks (one process per GPU).

The random states of the trace estimate are independent, and the paper
distributes them over MPI processes (Sec. 2.4.2). Here each rank propagates
its own shard of states with no communication on the data path; the only
exchange is the average of the per-state correlations (or moments) once at the
end, a few kilobytes, through torch.distributed (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations


def shard_states(nstates: int, rank: int, world: int) -> list[int]:
    """State indices owned by `rank`: j = rank, rank + world, ... (< nstates)."""
    if world < 1 or not (0 <= rank < world) or nstates < 0:
        raise ValueError("invalid shard request")
    return list(range(rank, nstates, world))


def average_over_ranks(local_sum, nstates: int, group=None):
    """Sum of the ranks' per-state results divided by the total state count.

    local_sum: torch tensor holding this rank's sum over its own states (any
    shape, real or complex); the tensor is reduced in place and returned."""
    import torch
    import torch.distributed as dist
    t = local_sum
    if t.is_complex():
        v = torch.view_as_real(t)
        dist.all_reduce(v, group=group)
    else:
        dist.all_reduce(t, group=group)
    return t / nstates

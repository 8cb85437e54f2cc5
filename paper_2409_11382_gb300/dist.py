"""Host-side logic of multi-GPU runs.

Instances of the solver never exchange data: a single instance is not split
across GPUs, and batched or served instances are sharded by instance.  So the
only collectives are on the host side of the benchmark -- a barrier and the
maximum of the per-rank timings -- and none sits on the data path.
"""
from __future__ import annotations

import os


def rank_world():
    """(rank, world size, local rank) from the torchrun environment (1 process if unset)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(count: int, rank: int, world: int) -> list:
    """Indices of the instances rank ``rank`` of ``world`` owns: round-robin, so that
    every instance has exactly one owner and the shards differ in size by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    return list(range(rank, count, world))


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a scalar over all ranks of the default process group (the value
    itself without one).  Works on the gloo (CPU) and nccl (GPU) backends."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())

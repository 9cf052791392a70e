"""Spreading independent migrations over ranks (one process per GPU).

The path has no exchange step: (velocity sample, shot) migrations are
independent, so ranks split the items and only the timing is combined.  The
paper hands such subgroups of migrations to MPI ranks (§3); here each rank
is one GPU.
"""
from __future__ import annotations


def shard(n_items: int, rank: int, world: int) -> list:
    """Round-robin share of items 0..n_items-1 for `rank` of `world`."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} of world {world}")
    return list(range(rank, n_items, world))


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """Largest value of x over all ranks (host-side, gloo or nccl)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())

"""Spreading independent migrations over ranks (one process per GPU).

(velocity sample, shot) migrations are independent, so ranks split the items
and, for throughput runs, only the timing is combined.  The paper hands such
subgroups of migrations to MPI ranks (§3); here each rank is one GPU.  The
ensemble statistics are the one step that needs data from every rank: see
the pixel-slab exchange below.
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


# ------------------------------------------------ sharded ensemble stats --
#
# The one real exchange of the path: a rank migrates a contiguous share of
# the velocity samples (whole images, no shot stacks to combine), but the
# per-pixel quantiles (§2.3) need every sample's value at a pixel.  An
# all-to-all hands each rank a contiguous pixel slab of all images, samples
# in global order, so the per-slab statistics equal the unsharded ones; the
# slabs of the results are then gathered.  Works on CPU tensors (gloo) and
# on CUDA tensors (nccl) alike.

def share(n: int, rank: int, world: int) -> tuple:
    """Contiguous share [start, end) of n items for `rank` of `world`."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} of world {world}")
    return n * rank // world, n * (rank + 1) // world


def to_pixel_slabs(local, nsample: int, rank: int, world: int):
    """This rank's images local [n_local][npix] (its share of the nsample
    samples, in order) -> [nsample][slab] for this rank's pixel slab."""
    npix = int(local.shape[-1])
    local = local.reshape(-1, npix)
    if world == 1:
        return local
    import torch
    import torch.distributed as dist

    shares = [share(nsample, r, world) for r in range(world)]
    slabs = [share(npix, r, world) for r in range(world)]
    n_local = shares[rank][1] - shares[rank][0]
    if local.shape[0] != n_local:
        raise ValueError(f"rank {rank} holds {local.shape[0]} images, its share is {n_local}")
    send = torch.cat([local[:, a:b].reshape(-1) for a, b in slabs])
    mine = slabs[rank][1] - slabs[rank][0]
    in_splits = [n_local * (b - a) for a, b in slabs]
    out_splits = [(e - s) * mine for s, e in shares]
    recv = torch.empty(sum(out_splits), dtype=local.dtype, device=local.device)
    dist.all_to_all_single(recv, send, out_splits, in_splits)
    return torch.cat([p.reshape(-1, mine) for p in torch.split(recv, out_splits)], 0)


def gather_slabs(x, npix: int, rank: int, world: int):
    """Every rank's pixel slab x (1-D) joined into the full [npix] array, on
    every rank."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    slabs = [share(npix, r, world) for r in range(world)]
    width = max(b - a for a, b in slabs)
    pad = torch.zeros(width, dtype=x.dtype, device=x.device)
    pad[:x.numel()] = x
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    return torch.cat([p[:b - a] for p, (a, b) in zip(parts, slabs)])


def sharded_ensemble_stats(local, nsample: int, rank: int, world: int, stats_fn):
    """Per-pixel (mean, std, q05, q95) of the whole ensemble from each rank's
    share of the images.  stats_fn(images [n][npix]) returns the four arrays
    of one slab (the library's rtm_ensemble_stats on the GPU)."""
    npix = int(local.shape[-1])
    slab = to_pixel_slabs(local, nsample, rank, world)
    return tuple(gather_slabs(s, npix, rank, world) for s in stats_fn(slab))

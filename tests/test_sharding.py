"""Multi-rank host logic on CPU: two gloo ranks split the migrations without
overlap or gaps and agree on the max-over-ranks timing."""
import os
import socket

import pytest

from paper_2001_06444_gb300.sharding import shard


def test_shard_partitions_items():
    for world in (1, 2, 3, 8):
        got = sorted(i for r in range(world) for i in shard(97, r, world))
        assert got == list(range(97))
    with pytest.raises(ValueError):
        shard(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist

    from paper_2001_06444_gb300.sharding import barrier, max_over_ranks, shard

    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard(96, rank, world)
    out = [None] * world
    dist.all_gather_object(out, mine)
    barrier(world)
    m = max_over_ranks(1.5 + rank, world)
    q.put((rank, out, m))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, m in res:
        assert m == 2.5
        flat = sorted(i for part in gathered for i in part)
        assert flat == list(range(96))
        assert not set(gathered[0]) & set(gathered[1])


def _stats_rank(rank, world, port, nsample, npix, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import numpy as np
    import torch
    import torch.distributed as dist

    from oracle.stats import ensemble_stats
    from paper_2001_06444_gb300 import inputs
    from paper_2001_06444_gb300.sharding import share, sharded_ensemble_stats, to_pixel_slabs

    dist.init_process_group("gloo", rank=rank, world_size=world)
    full = inputs.normal(77, nsample * npix).reshape(nsample, npix)
    a, b = share(nsample, rank, world)
    local = torch.from_numpy(full[a:b].copy())
    slab = to_pixel_slabs(local, nsample, rank, world)
    s0, s1 = share(npix, rank, world)
    slab_ok = bool(np.array_equal(slab.numpy(), full[:, s0:s1]))

    def cpu_stats(x):
        return tuple(torch.from_numpy(np.ascontiguousarray(v)) for v in ensemble_stats(x.numpy()))

    got = sharded_ensemble_stats(local, nsample, rank, world, cpu_stats)
    q.put((rank, slab_ok, [g.numpy() for g in got]))
    dist.destroy_process_group()


@pytest.mark.parametrize("world,nsample,npix", [(2, 7, 1001), (3, 10, 257)])
def test_sharded_ensemble_stats_equal_unsharded(world, nsample, npix):
    # ragged shares of samples and pixels; the statistics of every pixel come
    # out exactly as computed on the whole ensemble
    import numpy as np
    import torch.multiprocessing as mp

    from oracle.stats import ensemble_stats
    from paper_2001_06444_gb300 import inputs

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_stats_rank, args=(r, world, port, nsample, npix, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = ensemble_stats(inputs.normal(77, nsample * npix).reshape(nsample, npix))
    for rank, slab_ok, got in res:
        assert slab_ok
        for g, w in zip(got, want):
            assert np.array_equal(g, w)

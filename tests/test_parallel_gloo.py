"""Multi-rank host logic on CPU with the gloo backend (world size 2)."""
import os

import pytest
import torch.multiprocessing as mp

from paper_2406_11185_gb300 import parallel


def test_shard_molecules_partition():
    for nmol in (0, 1, 5, 256):
        for world in (1, 2, 3, 8):
            parts = [parallel.shard_molecules(nmol, r, world) for r in range(world)]
            flat = [i for p in parts for i in p]
            assert flat == list(range(nmol))
            assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        parallel.shard_molecules(4, 2, 2)


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = parallel.shard_molecules(10, rank, world)
        ms, units = parallel.aggregate(100.0 + 50.0 * rank, len(mine))
        q.put((rank, ms, units))
    finally:
        dist.destroy_process_group()


def test_aggregate_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, units in res:
        assert ms == 150.0          # the slowest rank
        assert units == 10.0        # every molecule counted once


def test_aggregate_without_process_group():
    assert parallel.aggregate(7.0, 3.0) == (7.0, 3.0)

"""Multi-rank host logic on CPU with the gloo backend (world size 2)."""
import os

import numpy as np
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


def test_assign_class_pairs_partition_and_balance():
    rng = np.random.default_rng(3)
    cost = rng.exponential(100.0, size=(2, 55))
    cost[rng.random((2, 55)) < 0.3] = 0.0  # empty class pairs
    for world in (1, 2, 3, 8):
        m = parallel.assign_class_pairs(cost, world)
        assert m.shape == (world, 2, 55)
        owned = m.sum(axis=0)
        assert np.all(owned[cost > 0] == 1) and np.all(owned[cost == 0] == 0)
        loads = np.array([(m[r] * cost).sum() for r in range(world)])
        # LPT: no rank exceeds the average by more than the largest single job
        assert loads.max() <= cost.sum() / world + cost.max() + 1e-9
        assert np.array_equal(m, parallel.assign_class_pairs(cost, world))  # deterministic
    with pytest.raises(ValueError):
        parallel.assign_class_pairs(-cost, 2)


def _shard_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank 0's costs decide; the other ranks pass different costs on purpose
        cost = np.arange(110, dtype=np.float64).reshape(2, 55) + (0.0 if rank == 0 else 1000.0 * rank)
        cost[:, ::7] = 0.0
        mask = parallel.class_pair_masks(cost, world, rank)
        # a stand-in for the per-class-pair partial results: contribution
        # (band * 55 + cp + 1) of every owned class pair, summed across ranks
        vals = np.arange(1, 111, dtype=np.float64).reshape(2, 55)
        part = torch.tensor([float((vals * mask).sum())], dtype=torch.float64)
        parallel.sum_partials(part)
        q.put((rank, mask.tolist(), float(part.item())))
    finally:
        dist.destroy_process_group()


def test_sharded_partials_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29700 + os.getpid() % 1000
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    res = sorted(q.get(timeout=10) for _ in range(2))
    m0, m1 = np.array(res[0][1]), np.array(res[1][1])
    cost0 = np.arange(110, dtype=np.float64).reshape(2, 55)
    cost0[:, ::7] = 0.0
    assert np.array_equal(np.stack([m0, m1]), parallel.assign_class_pairs(cost0, 2))  # rank 0's partition
    assert np.all(m0 + m1 == (cost0 > 0))
    vals = np.arange(1, 111, dtype=np.float64).reshape(2, 55)
    for _, _, total in res:
        assert total == float((vals * (cost0 > 0)).sum())  # every owned class pair summed once

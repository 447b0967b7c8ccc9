"""Multi-rank helpers (one process per GPU, torch.distributed).

Single molecule: the J/K build shards by class pair.  Each (band, class pair)
launch is independent work (its own quartets, its own work counter), so each
rank evaluates the class pairs of its mask (adft_opts.pair_mask) and holds
partial J, K, E or gradient; one sum all-reduce of those partials is the only
exchange.  The masks come from a longest-processing-time assignment of the
class pairs by their measured kernel times (adft_autotune), computed on rank 0
and broadcast, so that every rank uses the same partition.

Batched form: whole molecules are sharded across ranks with no data exchange.
The remaining collectives are on timing and counts: the slowest rank's time
and the total work of all ranks.
"""
from __future__ import annotations

import numpy as np

NCP = 55  # class pairs (l <= 3)


def shard_molecules(nmol: int, rank: int, world: int) -> list[int]:
    """Contiguous, balanced block of molecule indices owned by `rank`."""
    if world <= 0 or not (0 <= rank < world) or nmol < 0:
        raise ValueError("need world > 0, 0 <= rank < world, nmol >= 0")
    base, extra = divmod(nmol, world)
    start = rank * base + min(rank, extra)
    return list(range(start, start + base + (1 if rank < extra else 0)))


def assign_class_pairs(cost, world: int) -> np.ndarray:
    """Partition the (band, class pair) launches over `world` ranks.

    cost: [2, 55] non-negative costs (e.g. measured kernel ms; 0 = empty).
    Returns masks [world, 2, 55] of 0/1 in which every entry with cost > 0 is
    owned by exactly one rank and every empty entry by none: the longest
    processing time rule (largest first, onto the least loaded rank, ties to
    the lower rank), deterministic for a given cost table."""
    c = np.asarray(cost, dtype=np.float64).reshape(2, NCP)
    if world <= 0:
        raise ValueError("world must be > 0")
    if np.any(c < 0) or not np.all(np.isfinite(c)):
        raise ValueError("costs must be finite and >= 0")
    masks = np.zeros((world, 2, NCP), dtype=np.uint8)
    load = np.zeros(world)
    order = sorted(((c[b, p], b, p) for b in range(2) for p in range(NCP) if c[b, p] > 0),
                   key=lambda t: (-t[0], t[1], t[2]))
    for w, b, p in order:
        r = int(np.argmin(load))
        masks[r, b, p] = 1
        load[r] += w
    return masks


def class_pair_masks(cost, world: int, rank: int, device=None) -> np.ndarray:
    """This rank's [2, 55] mask: rank 0 assigns from its cost table and
    broadcasts, so every rank holds the same partition (the identity mask of
    rank 0's assignment without a process group)."""
    import torch
    import torch.distributed as dist
    masks = assign_class_pairs(cost, world) if rank == 0 else np.zeros((world, 2, NCP), dtype=np.uint8)
    if dist.is_available() and dist.is_initialized() and world > 1:
        t = torch.from_numpy(masks.astype(np.int32)).to(device)
        dist.broadcast(t, src=0)
        masks = t.cpu().numpy().astype(np.uint8)
    return masks[rank]


def sum_partials(*tensors):
    """In-place sum all-reduce of the partial results (J, K, E or gradient):
    the one exchange step of the sharded build.  No-op without a process group."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        for t in tensors:
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return tensors


def aggregate(ms_total: float, units: float, device=None) -> tuple[float, float]:
    """(max of ms_total over ranks, sum of units over ranks); the identity
    without an initialised process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(ms_total), float(units)
    t = torch.tensor([float(ms_total)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())

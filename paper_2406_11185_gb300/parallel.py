"""Multi-rank helpers (one process per GPU, torch.distributed).

The single-molecule J/K build runs as independent replicas, one per rank; the
batched form shards whole molecules across ranks with no data exchange.  The
only collectives are on the host-visible timing and counts: the slowest rank's
time and the total work of all ranks.
"""
from __future__ import annotations


def shard_molecules(nmol: int, rank: int, world: int) -> list[int]:
    """Contiguous, balanced block of molecule indices owned by `rank`."""
    if world <= 0 or not (0 <= rank < world) or nmol < 0:
        raise ValueError("need world > 0, 0 <= rank < world, nmol >= 0")
    base, extra = divmod(nmol, world)
    start = rank * base + min(rank, extra)
    return list(range(start, start + base + (1 if rank < extra else 0)))


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

"""Host-side logic of running the solver on several GPUs.

Keyframes (and camera streams) are independent problems, so N GPUs run N
replicas that each own a share of the work; nothing on the data path crosses
GPUs. The only cross-rank steps are the bookkeeping of a benchmark or a
server: which rank owns which item, and the max / sum of per-rank timings
and counts (over torch.distributed, any backend).
"""
from __future__ import annotations

from typing import List


def shard(n_items: int, rank: int, world: int) -> List[int]:
    """Items owned by `rank`: a contiguous, balanced block (sizes differ by at
    most one); every item is owned by exactly one rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    if n_items < 0:
        raise ValueError("n_items < 0")
    lo = n_items * rank // world
    hi = n_items * (rank + 1) // world
    return list(range(lo, hi))


def rank_seed(base: int, rank: int) -> int:
    """Seed of a rank's own synthetic workload (weak scaling: each rank solves
    a different scene of the same shape)."""
    return base + 1000 * rank


def _reduce(x: float, op: str, device=None) -> float:
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(x: float, device=None) -> float:
    """Largest value over all ranks (the job's time is its slowest rank's)."""
    return _reduce(x, "max", device)


def sum_over_ranks(x: float, device=None) -> float:
    return _reduce(x, "sum", device)

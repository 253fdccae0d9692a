"""Island sharding over ranks: the islands are independent (the paper's
recording simulations run as independent jobs, Sec. II.C), so N GPUs run N
replicas of the batched path on disjoint island ranges with no collective on
the data path; only the timed region's duration is reduced (max over ranks)."""
from __future__ import annotations


def island_range(islands_per_rank: int, rank: int) -> tuple[int, int]:
    """[first, last) global island indices of one rank (weak scaling)."""
    if islands_per_rank < 1 or rank < 0:
        raise ValueError("islands_per_rank >= 1 and rank >= 0 required")
    return rank * islands_per_rank, (rank + 1) * islands_per_rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest value over all ranks (the job's time is its slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())

"""Data-parallel sharding of a batch of machines over ranks.

The machines of a batch are independent (the map Phi of Sec. 2 acts on each
configuration separately), so ranks exchange nothing while they run: rank r
owns the contiguous VM range [r * per_rank, (r + 1) * per_rank) of the
workload, generated from the same counter-based generator, and the only
communication is the reduction of the timing and the counts at the end.
"""
from __future__ import annotations


def shard_range(rank: int, per_rank: int) -> tuple[int, int]:
    """First VM id and VM count of `rank`'s shard (weak scaling: a fixed
    number of VMs per rank)."""
    if rank < 0 or per_rank <= 0:
        raise ValueError("rank must be >= 0 and per_rank > 0")
    return rank * per_rank, per_rank


def combine(dist, elapsed_ms: float, vm_steps: int, device=None) -> tuple[float, int]:
    """Whole-job (max elapsed ms over ranks, total VM-steps over ranks).
    `dist` is torch.distributed with an initialised process group, or None
    for a single process."""
    if dist is None:
        return float(elapsed_ms), int(vm_steps)
    import torch
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    n = torch.tensor([int(vm_steps)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(n.item())

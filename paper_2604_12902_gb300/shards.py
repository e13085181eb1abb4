"""Data-parallel sharding of a batch of machines over ranks.

The machines of a batch are independent (the map Phi of Sec. 2 acts on each
configuration separately), so ranks exchange nothing while they run: rank r
owns the contiguous VM range [r * per_rank, (r + 1) * per_rank) of the
workload, generated from the same counter-based generator, and the only
communication is the reduction of the timing and the counts at the end.
A fixed batch can instead be split into contiguous ranges of balanced
estimated cost (``balanced_ranges``), so that no rank gets most of the
long-running machines.
"""
from __future__ import annotations


def shard_range(rank: int, per_rank: int) -> tuple[int, int]:
    """First VM id and VM count of `rank`'s shard (weak scaling: a fixed
    number of VMs per rank)."""
    if rank < 0 or per_rank <= 0:
        raise ValueError("rank must be >= 0 and per_rank > 0")
    return rank * per_rank, per_rank


def estimated_cost(wl) -> "np.ndarray":
    """Work estimate per VM for balancing shards: its step cap (an upper
    bound on the VM-steps it can take), so that ranks holding long-running
    VMs get fewer of them."""
    import numpy as np
    return np.minimum(np.asarray(wl.caps, np.uint64), np.uint64(1 << 40)).astype(np.int64)


def balanced_ranges(costs, ranks: int) -> list[tuple[int, int]]:
    """Split VMs 0..V-1 into `ranks` contiguous ranges (first, count), in
    rank order, so that the largest range cost (sum of `costs` over the
    range) is as small as possible. Binary search on that bound with a greedy
    check: for a bound B, each range takes VMs while its cost stays <= B, and
    B is feasible when at most `ranks` ranges cover the batch. Ranks beyond
    the number of ranges needed get empty ranges at the end."""
    import numpy as np
    c = np.asarray(costs, np.int64)
    if ranks <= 0:
        raise ValueError("ranks must be > 0")
    if (c < 0).any():
        raise ValueError("costs must be >= 0")
    V = int(c.shape[0])
    pre = np.concatenate([[0], np.cumsum(c)])

    def cuts(bound):
        out, start = [], 0
        while start < V and len(out) < ranks:
            # last end e with pre[e] - pre[start] <= bound, at least one VM
            e = int(np.searchsorted(pre, pre[start] + bound, side="right")) - 1
            e = max(e, start + 1)
            out.append((start, e - start))
            start = e
        return out, start >= V

    lo, hi = int(c.max()) if V else 0, int(pre[-1])
    while lo < hi:
        mid = (lo + hi) // 2
        if cuts(mid)[1]:
            hi = mid
        else:
            lo = mid + 1
    ranges, _ = cuts(lo)
    end = ranges[-1][0] + ranges[-1][1] if ranges else 0
    ranges += [(end, 0)] * (ranks - len(ranges))
    return ranges


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


def combine_counts(dist, counts, device=None):
    """Element-wise sum over ranks of a small integer array (a tau_h
    histogram, status counts): the only other exchange the sharded path has.
    `dist` as for combine; returns a numpy int64 array."""
    import numpy as np
    a = np.asarray(counts, np.int64)
    if dist is None:
        return a.copy()
    import torch
    t = torch.as_tensor(a, device=device).clone()
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().numpy()

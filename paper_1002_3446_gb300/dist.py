"""Event-range sharding across ranks and the one exchange of the path.

Events are independent functions of (seed, event index), so rank r of W
generates the disjoint range [first + r N, first + (r+1) N) and no data moves
during generation.  The only exchange is the sum of the accumulators
(sum w, sum w^2, n_pass, n_generated, their compensation terms, n_nonfinite)
and of the histogram bins, once at the end: a few hundred bytes.
"""
from __future__ import annotations


def event_range(rank, world, n_per_rank, first=0):
    """First event and count of `rank`'s shard (weak scaling: N per rank)."""
    if not (0 <= rank < world):
        raise ValueError("rank outside 0..world-1")
    return first + rank * n_per_rank, n_per_rank


def reduce_sums(*tensors, group=None):
    """Sum accumulator / histogram tensors over all ranks (in place).  Works for
    any torch.distributed backend (gloo on CPU tensors, nccl on CUDA ones)."""
    import torch.distributed as dist
    for t in tensors:
        if t is not None:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return tensors


def sigma_from_acc(acc):
    """Cross section and MC error (pb) from a reduced accumulator vector."""
    import math
    n = float(acc[3])
    sw = float(acc[0]) + float(acc[4])
    sw2 = float(acc[1]) + float(acc[5])
    mean = sw / n if n > 0 else 0.0
    var = (sw2 / n - mean * mean) / (n - 1) if n > 1 else 0.0
    return mean, math.sqrt(max(var, 0.0))

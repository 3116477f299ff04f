"""Multi-process layout: one process per GPU, independent problems.

Fits are independent, so the batch shards across ranks with no collective on
the data path; the only collectives are a barrier around the timed region and
the max of the step times (so the slowest rank sets the job time).
"""
from __future__ import annotations


def shard_range(B: int, rank: int, world: int) -> tuple:
    """Contiguous share [lo, hi) of B problems for `rank` of `world`;
    sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world or B < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(B, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Largest `value` over the ranks of the default process group (the
    value itself without one)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())

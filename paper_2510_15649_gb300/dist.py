"""Multi-process layout: one process per GPU, independent problems.

Fits are independent, so a batch shards across ranks with no collective on
the data path (by problem count or by cost, contiguous shares), and serving
requests are routed to per-GPU slot pools by load (route_requests); the only
collectives are a barrier around the timed region, the max of the step
times (so the slowest rank sets the job time) and sums or gathers of
counts and latencies for the report.
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


def cost_shard_range(cost, rank: int, world: int) -> tuple:
    """Contiguous share [lo, hi) of the problems for `rank` of `world`,
    balanced by per-problem cost (e.g. problem_cost, the work a fit does
    along its path): rank r's share ends at the prefix whose running cost
    is nearest to (r + 1) / world of the total, so every boundary is within
    half a problem's cost of its target and every rank's cost within one
    problem's cost of total / world.  Contiguous shares keep every rank's
    problems one slice of the offsets."""
    import numpy as np
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad shard arguments")
    c = np.asarray(cost, np.float64)
    if c.ndim != 1 or np.any(c < 0) or not np.all(np.isfinite(c)):
        raise ValueError("costs must be a finite non-negative vector")
    B = len(c)
    if B == 0:
        return 0, 0
    cum = np.cumsum(c)
    total = cum[-1]
    if total <= 0:
        return shard_range(B, rank, world)

    def end(r):  # the prefix length whose running cost is nearest the target
        if r == world - 1:
            return B
        t = total * (r + 1) / world
        k = int(np.searchsorted(cum, t, side="left"))  # cum[k] >= t > cum[k-1]
        below = cum[k - 1] if k > 0 else 0.0
        return k + 1 if cum[k] - t < t - below else k

    lo = 0 if rank == 0 else min(end(rank - 1), B)
    hi = max(lo, min(end(rank), B))
    return lo, hi


def shard_batch(batch: dict, lo: int, hi: int) -> dict:
    """Problems lo..hi-1 of a batch (the layout of `synth`) as a batch of
    their own: the same shared X, their slots of y / row_idx, offsets
    rebased to start at 0."""
    import numpy as np
    off = np.asarray(batch["offsets"], np.int64)
    a, b = int(off[lo]), int(off[hi])
    ri = batch.get("row_idx")
    out = dict(batch)
    out.update(y=batch["y"][a:b], offsets=off[lo:hi + 1] - a,
               p=np.asarray(batch["p"])[lo:hi])
    if ri is None:
        out["X"] = batch["X"][a:b]  # slots are rows of X
        out["row_idx"] = None
    else:
        out["row_idx"] = ri[a:b]
    return out


STEP_ROWS = 1024  # a 1-D step's fixed work (window sums, selection), in rows


def problem_cost(batch: dict, L: int) -> "np.ndarray":
    """Estimated work of each problem's fit along an L-point path,
    p * (n + STEP_ROWS) * L: about p 1-D steps per sweep, each a pass over
    the n rows plus a fixed part worth about a thousand rows (the estimate
    the fit kernels' longest-first work order uses)."""
    import numpy as np
    n = np.diff(np.asarray(batch["offsets"], np.int64)).astype(np.float64)
    return np.asarray(batch["p"], np.float64) * (n + STEP_ROWS) * L


def cost_share(batch: dict, L: int, rank: int, world: int) -> tuple:
    """This rank's share of one batch for strong scaling: contiguous
    problems balanced by problem_cost (cost_shard_range), cut out with
    shard_batch.  Returns (the share as a batch, (lo, hi))."""
    lo, hi = cost_shard_range(problem_cost(batch, L), rank, world)
    return shard_batch(batch, lo, hi), (lo, hi)


def covered_once(lo: int, hi: int, B: int, dist=None, device=None) -> bool:
    """True when the ranks' shares [lo, hi) of B problems cover every
    problem exactly once (a sum over ranks of each rank's indicator)."""
    import torch
    t = torch.zeros(B, dtype=torch.int32, device=device if device is not None else "cpu")
    t[lo:hi] = 1
    if dist is not None and dist.is_available() and dist.is_initialized():
        dist.all_reduce(t)
    return bool(torch.all(t == 1).item())


def route_requests(sizes, world: int) -> "np.ndarray":
    """Rank (GPU) for each serving request, in arrival order: the rank with
    the least work routed to it so far (ties to the lowest rank), the work
    of a request being its size (e.g. n * p, the design it fits along its
    path).  Deterministic, so every rank computes the same routing from the
    same trace with no exchange; each rank then serves its own requests in
    its own slot pool."""
    import numpy as np
    if world < 1:
        raise ValueError("bad world size")
    w = np.asarray(sizes, np.float64)
    if w.ndim != 1 or np.any(w < 0) or not np.all(np.isfinite(w)):
        raise ValueError("sizes must be a finite non-negative vector")
    load = np.zeros(world)
    out = np.empty(len(w), np.int64)
    for i, c in enumerate(w):
        r = int(np.argmin(load))
        out[i] = r
        load[r] += c
    return out


def gather_lists(values: list, dist=None) -> list:
    """Concatenation, in rank order, of every rank's list (the list itself
    without a process group); host objects, for statistics."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return list(values)
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, list(values))
    return [v for part in parts for v in part]


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


def sum_over_ranks(value: float, dist=None, device=None) -> float:
    """Sum of `value` over the ranks of the default process group (the
    value itself without one): work counted on every rank."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())

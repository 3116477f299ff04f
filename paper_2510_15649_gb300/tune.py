"""Autotuner for the batched fit's launch shape.

The fit kernel has four shapes (a group of 32, 64 or 128 threads per fit
with several fits per thread block, or one 512-thread block per fit) and,
for the small groups, a number of fits per block bounded by shared memory; problems are taken
longest first or longest and shortest alternately.  More fits per block
hide more latency but also keep more gathered designs live in L2 at once,
so the best choice depends on the problem mix.  `autotune` times every
candidate on an evenly strided sample of the problem set (same size mix)
with CUDA events and returns the fastest; choices are cached per device,
problem-set signature and options (`cache_key`).  Per-fit results do not depend on fits_per_block;
the two shapes agree within the float32 tolerance.
"""
from __future__ import annotations

import numpy as np
import torch

from . import ladlasso as ll

_cache: dict = {}


def save_cache(path: str) -> None:
    """Write the autotuner's choices (per device and problem-set signature)
    to a JSON file."""
    import json
    rows = [{"key": list(k), "choice": [c.group_threads, c.fits_per_block, c.work_order],
             "seconds": {f"{x.group_threads}x{x.fits_per_block}/o{x.work_order}": t
                         for x, t in times.items()}}
            for k, (c, times) in _cache.items()]
    with open(path, "w") as f:
        json.dump(rows, f, indent=1)


def load_cache(path: str) -> int:
    """Read choices written by save_cache; returns how many were loaded."""
    import json
    with open(path) as f:
        rows = json.load(f)
    for r in rows:
        g, fb, o = r["choice"]
        times = {}
        for tag, t in r.get("seconds", {}).items():
            gs, rest = tag.split("x")
            fs, os_ = rest.split("/o")
            times[ll.Launch(int(gs), int(fs), int(os_))] = float(t)
        _cache[tuple(r["key"])] = (ll.Launch(g, fb, o), times)
    return len(rows)


def cache_key(pr: ll.Problems, L: int, opts: ll.Opts | None = None, device_name: str = "") -> tuple:
    """Signature under which a choice is cached (flat, so it survives the
    JSON file): device, problem-set shape (P, n_max, B, path length, total
    rows, row-index layout) and every method option, which all change the
    work per fit."""
    o = opts if opts is not None else ll.default_opts()
    return (device_name, pr.P, pr.n_max, pr.B, L, pr.row_idx is None, int(pr.y.numel()),
            *(getattr(o, f) for f, _ in o._fields_))


def candidates(pr: ll.Problems) -> list:
    """Launch shapes the library accepts for `pr`: groups of 32, 64 or 128
    threads per fit with the most fits per block that shared memory holds
    and down to a third of that, and one 512-thread block per fit; each in
    both work orders."""
    out = []
    for gt in (32, 64, 128):
        g, fmax, mrows = ll.launch_shape(pr, ll.Launch(gt, 0))
        if pr.n_max > mrows:
            continue
        lo = max(1, fmax // 3)
        for order in (0, 1):
            out += [ll.Launch(gt, f, order) for f in range(fmax, lo - 1, -1)]
    g, _, mrows = ll.launch_shape(pr, ll.Launch(512, 0))
    if pr.n_max <= mrows:
        out += [ll.Launch(512, 0, 0), ll.Launch(512, 0, 1)]
    return out


def _subset(pr: ll.Problems, lambdas: torch.Tensor, every: int):
    """Every `every`-th problem of pr as its own problem set (device copies)."""
    off = pr.offsets.cpu().numpy()
    qs = np.arange(0, pr.B, every)
    lens = off[qs + 1] - off[qs]
    idx = np.concatenate([np.arange(off[q], off[q + 1]) for q in qs]) if len(qs) else np.zeros(0, np.int64)
    dev = pr.X.device
    idx_t = torch.as_tensor(idx, device=dev)
    qs_t = torch.as_tensor(qs, device=dev)
    new_off = torch.as_tensor(np.concatenate([[0], np.cumsum(lens)]).astype(np.int64), device=dev)
    y = pr.y[idx_t]
    if pr.row_idx is None:
        X, row_idx = pr.X[idx_t], None
    else:
        X, row_idx = pr.X, pr.row_idx[idx_t]
    sub = ll.Problems(X=X, y=y, offsets=new_off, row_idx=row_idx,
                      p=None if pr.p is None else pr.p[qs_t], P=pr.P, n_max=pr.n_max,
                      n_rows=None if pr.n_rows is None else pr.n_rows[qs_t])
    return sub, lambdas.reshape(pr.B, -1)[qs_t].contiguous()


def autotune(pr: ll.Problems, lambdas: torch.Tensor, *, opts: ll.Opts | None = None,
             sample_problems: int = 512, repeats: int = 2, use_cache: bool = True,
             tie: float = 0.01) -> tuple:
    """Fastest launch shape for fitting `pr` along `lambdas`; among shapes
    within `tie` (relative) of the fastest, the one-warp shape with the fewest
    fits per block (smaller instruction-cache and L2 footprint per SM).
    Returns (Launch, {shape: seconds})."""
    L = int(lambdas.reshape(pr.B, -1).shape[1])
    dev = pr.X.device
    key = cache_key(pr, L, opts, torch.cuda.get_device_name(dev))
    if use_cache and key in _cache:
        return _cache[key]
    cands = candidates(pr)
    if not cands:
        raise ll.LadLassoError("no launch shape holds problems of n_max rows")
    every = max(1, pr.B // max(1, sample_problems))
    sub, lam = _subset(pr, lambdas, every) if every > 1 else (pr, lambdas)
    ws = ll.workspace(sub, L)
    stream = torch.cuda.current_stream(dev)
    times = {}
    for c in cands:
        ll.fit(sub, lam, ws=ws, opts=opts, launch=c)  # warm-up
        best = float("inf")
        for _ in range(repeats):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ll.fit(sub, lam, ws=ws, opts=opts, launch=c)
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        times[c] = best
    choice = choose(times, tie)
    _cache[key] = (choice, times)
    return choice, times


def choose(times: dict, tie: float = 0.01):
    """The shape to use given measured seconds per shape: among shapes
    within `tie` (relative) of the fastest, the smallest group of threads
    per fit, then the fewest fits per block, then work order 0."""
    best = min(times.values())
    near = [c for c, t in times.items() if t <= best * (1.0 + tie)]
    return min(near, key=lambda c: (c.group_threads, c.fits_per_block, c.work_order))

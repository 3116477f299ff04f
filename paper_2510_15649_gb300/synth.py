"""Seeded synthetic inputs for batched LAD-LASSO fits.

This module draws random numbers and lays them out; it holds none of the
method's arithmetic (no objective, no lambda_max, no fitting). Both the CPU
oracle tests and the CUDA path take their inputs from here.

The paper (Section 4) draws its data with a make-regression style generator
(1-5 explanatory variables, 10-30 points). The workloads below keep that
structure -- a sparse true coefficient vector, Gaussian design, heavy-tailed
noise and shifted outlier rows -- at the sizes the batched path is built for:

  tiny      n=40, p=4, one fit, lambda=2                      (seed 0)
  batched   4096 row subsets of a shared 2000x32 X, uneven n, p (seed 1)
  large     256 fits, n=20000, p=128, AR(1) columns           (seed 2)
  diff      512 fits, n=500 (400 train / 100 validation), p=16 (seed 3)
  serve     Poisson arrivals, log-uniform n and p             (seed 4)

Layout handed to both sides (one "batch"):
  X        float32 [R, P] row-major, the shared design rows
  y        float32 [T]    targets, one per (problem, row) slot
  row_idx  int32   [T]    row of X used by slot t, or None when slots are X rows
  offsets  int64   [B+1]  problem b owns slots offsets[b] .. offsets[b+1]-1
  p        int32   [B]    problem b uses the leading p[b] columns of X
"""
from __future__ import annotations

import numpy as np

__all__ = ["tiny", "batched", "large", "diff", "serve_trace", "batched_like"]


def tiny(seed: int = 0) -> dict:
    """Single fit, n=40, p=4, b_true=[1.5,0,-2,0], Laplace(0,0.5) noise,
    4 rows (10%) shifted by +10, lambda=2.0."""
    rng = np.random.default_rng(seed)
    n, p = 40, 4
    X = rng.standard_normal((n, p))
    b_true = np.array([1.5, 0.0, -2.0, 0.0])
    noise = rng.laplace(0.0, 0.5, n)
    out = rng.choice(n, 4, replace=False)
    y = X @ b_true + noise
    y[out] += 10.0
    X = X.astype(np.float32)
    y = y.astype(np.float32)
    return dict(X=X, y=y, row_idx=None,
                offsets=np.array([0, n], np.int64), p=np.array([p], np.int32),
                lam=np.float32(2.0), b_true=b_true)


def batched_like(B: int, n_lo: int, n_hi: int, p_lo: int, p_hi: int,
                 R: int = 2000, P: int = 32, seed: int = 1) -> dict:
    """B problems, each a sorted random row subset (without replacement) of
    a shared R x P N(0,1) matrix, n ~ U{n_lo..n_hi}, p ~ U{p_lo..p_hi}
    leading columns, 3-sparse b_true ~ U(-3,3) at positions < p,
    Student-t(nu=2) noise.  Draw order: X, then per problem n, p, rows,
    support, values, noise."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((R, P)).astype(np.float32)
    ns = np.empty(B, np.int64)
    ps = np.empty(B, np.int32)
    rows, ys = [], []
    for b in range(B):
        n = int(rng.integers(n_lo, n_hi + 1))
        p = int(rng.integers(p_lo, p_hi + 1))
        r = np.sort(rng.choice(R, n, replace=False)).astype(np.int32)
        k = min(3, p)
        sup = rng.choice(p, k, replace=False)
        bt = np.zeros(p)
        bt[sup] = rng.uniform(-3.0, 3.0, k)
        noise = rng.standard_t(2.0, n)
        yb = X[r, :p].astype(np.float64) @ bt + noise
        ns[b], ps[b] = n, p
        rows.append(r)
        ys.append(yb.astype(np.float32))
    offsets = np.zeros(B + 1, np.int64)
    offsets[1:] = np.cumsum(ns)
    return dict(X=X, y=np.concatenate(ys), row_idx=np.concatenate(rows),
                offsets=offsets, p=ps)


def batched(B: int = 4096, seed: int = 1) -> dict:
    """Row subsets of a shared 2000x32 X, n in [50,2000], p in [4,32]."""
    return batched_like(B, 50, 2000, 4, 32, seed=seed)


def large(B: int = 256, n: int = 20000, p: int = 128, seed: int = 2) -> dict:
    """B contiguous problems of n rows x p columns; each row is an AR(1)
    sequence across columns with rho=0.5 (x_0 ~ N(0,1),
    x_j = rho x_{j-1} + sqrt(1-rho^2) e_j); b_true has 10 nonzeros ~ N(0, 4);
    Laplace(0,1) noise; 5% of rows get y += 20."""
    rng = np.random.default_rng(seed)
    rho = 0.5
    X = np.empty((B * n, p), np.float32)
    ys = np.empty(B * n, np.float32)
    s = np.sqrt(1.0 - rho * rho)
    for b in range(B):
        e = rng.standard_normal((n, p)).astype(np.float32)
        Xb = X[b * n:(b + 1) * n]
        Xb[:, 0] = e[:, 0]
        for j in range(1, p):
            Xb[:, j] = rho * Xb[:, j - 1] + s * e[:, j]
        sup = rng.choice(p, 10, replace=False)
        bt = np.zeros(p)
        bt[sup] = rng.normal(0.0, 2.0, 10)
        yb = Xb.astype(np.float64) @ bt + rng.laplace(0.0, 1.0, n)
        out = rng.choice(n, n // 20, replace=False)
        yb[out] += 20.0
        ys[b * n:(b + 1) * n] = yb
    offsets = np.arange(B + 1, dtype=np.int64) * n
    return dict(X=X, y=ys, row_idx=None, offsets=offsets,
                p=np.full(B, p, np.int32))


def diff(B: int = 512, n: int = 500, n_train: int = 400, p: int = 16,
         seed: int = 3) -> dict:
    """B problems with their own rows: X ~ N(0,1), 4-sparse b_true ~ U(-3,3),
    Laplace(0,1) noise. The first n_train rows of each problem are the
    training rows, the rest validation rows.  Returned as two batches
    (train, val) that share the same problem order."""
    rng = np.random.default_rng(seed)
    Xtr = np.empty((B * n_train, p), np.float32)
    Xva = np.empty((B * (n - n_train), p), np.float32)
    ytr = np.empty(B * n_train, np.float32)
    yva = np.empty(B * (n - n_train), np.float32)
    nv = n - n_train
    for b in range(B):
        X = rng.standard_normal((n, p))
        sup = rng.choice(p, 4, replace=False)
        bt = np.zeros(p)
        bt[sup] = rng.uniform(-3.0, 3.0, 4)
        y = X @ bt + rng.laplace(0.0, 1.0, n)
        Xtr[b * n_train:(b + 1) * n_train] = X[:n_train]
        Xva[b * nv:(b + 1) * nv] = X[n_train:]
        ytr[b * n_train:(b + 1) * n_train] = y[:n_train]
        yva[b * nv:(b + 1) * nv] = y[n_train:]
    return dict(train=dict(X=Xtr, y=ytr, row_idx=None,
                           offsets=np.arange(B + 1, dtype=np.int64) * n_train,
                           p=np.full(B, p, np.int32)),
                val=dict(X=Xva, y=yva, row_idx=None,
                         offsets=np.arange(B + 1, dtype=np.int64) * nv,
                         p=np.full(B, p, np.int32)))


def serve_trace(rate: float = 20000.0, seconds: float = 10.0, seed: int = 4,
                n_lo: int = 20, n_hi: int = 5000, p_lo: int = 2, p_hi: int = 64,
                max_requests: int | None = None, bank_rows: int | None = None) -> list:
    """Poisson arrivals (exponential gaps) at `rate` per second for `seconds`;
    each request is one fit with n log-uniform in [n_lo, n_hi] and p
    log-uniform in [p_lo, p_hi] (rounded), X ~ N(0,1), 3-sparse b_true
    ~ U(-3,3), Laplace(0,1) noise and 10% of rows shifted by +10.
    With `bank_rows`, each request's X is a window of n consecutive rows
    and its first p columns of one shared N(0,1) bank of bank_rows x p_hi
    (a view, so a long trace holds the bank, not a copy per request: 10 s
    at 20k requests/s would otherwise hold about 13 GB); its coefficients,
    noise and outliers are its own.
    Returns a list of dicts (t_arrival, X [n,p] float32, y [n] float32)."""
    rng = np.random.default_rng(seed)
    bank = None
    if bank_rows is not None:
        if bank_rows < n_hi:
            raise ValueError("the bank must hold the longest request")
        bank = rng.standard_normal((bank_rows, p_hi), dtype=np.float32)
    reqs = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= seconds:
            break
        if max_requests is not None and len(reqs) >= max_requests:
            break
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        p = int(round(np.exp(rng.uniform(np.log(p_lo), np.log(p_hi)))))
        if bank is None:
            X = rng.standard_normal((n, p))
        else:
            o = int(rng.integers(0, bank_rows - n + 1))
            X = bank[o:o + n, :p]
        k = min(3, p)
        sup = rng.choice(p, k, replace=False)
        bt = np.zeros(p)
        bt[sup] = rng.uniform(-3.0, 3.0, k)
        y = X @ bt + rng.laplace(0.0, 1.0, n)
        out = rng.choice(n, max(1, n // 10), replace=False)
        y[out] += 10.0
        reqs.append(dict(t=t, X=X if bank is not None else X.astype(np.float32),
                         y=y.astype(np.float32)))
    return reqs

"""Choosing lambda by cross-validation on held-out rows.

The paper picks the regularisation on data held out from the fit (Sections
2 and 6, with row subsets drawn combinatorially).  This driver runs that
selection as one batched workload on the library's kernels: every split is
one problem (its training rows as a row-index subset of the data), all
splits share one lambda path from lambda_max of the full data down to
ratio * lambda_max, the whole path of every split is fitted in one launch
(warm starts along the path), and ladlasso_path_loss evaluates the LAD
loss of every (split, lambda) on the split's held-out rows.  The host only
builds the index arrays and takes the argmin of the mean held-out loss.
Several data sets can be cross-validated in one launch (`cross_validate_many`).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import ladlasso as ll


@dataclass
class CVResult:
    """Cross-validation of one data set along its lambda path."""
    lambdas: np.ndarray    # [L] shared path
    loss: np.ndarray       # [S, L] held-out LAD loss per split
    mean_loss: np.ndarray  # [L] mean over splits of the per-row held-out loss
    best: int              # path position with the smallest mean loss
    b: np.ndarray          # [S, L, p] fitted coefficients per split
    status: np.ndarray     # [S, L]

    @property
    def best_lambda(self) -> float:
        """The lambda with the smallest mean held-out loss."""
        return float(self.lambdas[self.best])


def kfold_splits(n: int, K: int, seed: int = 0) -> list:
    """K disjoint held-out folds of a seeded permutation of the n rows;
    returns [(train_rows, heldout_rows)] with sorted row indices.
    2 <= K <= n, so that every fold holds rows out and keeps rows to fit."""
    if not 2 <= K <= n:
        raise ValueError(f"K-fold needs 2 <= K <= n (K = {K}, n = {n})")
    perm = np.random.default_rng(seed).permutation(n)
    folds = np.array_split(perm, K)
    return [(np.sort(np.concatenate(folds[:k] + folds[k + 1:])), np.sort(folds[k]))
            for k in range(K)]


def subset_splits(n: int, m: int, S: int, seed: int = 0) -> list:
    """S random leave-m-out splits (m held-out rows each, drawn without
    replacement within a split); 1 <= m < n."""
    if not 1 <= m < n or S < 1:
        raise ValueError(f"leave-m-out needs 1 <= m < n and S >= 1 (m = {m}, n = {n}, S = {S})")
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(S):
        ho = np.sort(rng.choice(n, m, replace=False))
        mask = np.ones(n, bool)
        mask[ho] = False
        out.append((np.nonzero(mask)[0], ho))
    return out


def _problem_set(X: torch.Tensor, y_rows: list, rows: list, P: int, p: int) -> ll.Problems:
    """Problems whose rows are the given row-index arrays of X."""
    dev = X.device
    lens = [len(r) for r in rows]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    ri = np.concatenate(rows).astype(np.int32) if rows else np.zeros(0, np.int32)
    y = torch.cat(y_rows) if y_rows else torch.zeros(0, device=dev)
    return ll.Problems(X=X, y=y, offsets=torch.as_tensor(off, device=dev),
                       row_idx=torch.as_tensor(ri, device=dev),
                       p=torch.full((len(rows),), p, dtype=torch.int32, device=dev), P=P,
                       n_max=int(max(lens)) if lens else 0)


def cross_validate_many(data: list, splits: list, L: int = 16, ratio: float = 1e-3,
                        opts: ll.Opts | None = None, device="cuda") -> list:
    """data: [(X [n, p] float32, y [n] float32)], splits: per data set a list
    of (train_rows, heldout_rows).  One fit launch and one loss launch for
    all splits of all data sets.  Returns [CVResult]."""
    dev = torch.device(device)
    P = max(int(np.asarray(X).shape[1]) for X, _ in data)
    # stack the data sets' rows into one design (zero-padded to P columns)
    Xs, ys, base = [], [], [0]
    for X, y in data:
        X = np.asarray(X, np.float32)
        Xp = np.zeros((X.shape[0], P), np.float32)
        Xp[:, :X.shape[1]] = X
        Xs.append(Xp)
        ys.append(np.asarray(y, np.float32))
        base.append(base[-1] + X.shape[0])
    Xd = torch.as_tensor(np.concatenate(Xs), device=dev)
    yd = torch.as_tensor(np.concatenate(ys), device=dev)
    # lambda_max of each full data set (one problem per data set)
    full = ll.Problems(X=Xd, y=yd,
                       offsets=torch.as_tensor(np.array(base, np.int64), device=dev),
                       p=torch.as_tensor(np.array([np.asarray(X).shape[1] for X, _ in data],
                                                  np.int32), device=dev),
                       P=P, n_max=max(b1 - b0 for b0, b1 in zip(base[:-1], base[1:])))
    lmax = ll.lambda_max(full)
    path = ll.lambda_path(lmax, L, ratio)  # [D, L]
    tr_rows, ho_rows, tr_y, ho_y, lam_rows, owner = [], [], [], [], [], []
    for d, ((X, _), sp) in enumerate(zip(data, splits)):
        for tr, ho in sp:
            tr_rows.append(np.asarray(tr) + base[d])
            ho_rows.append(np.asarray(ho) + base[d])
            tr_y.append(yd[torch.as_tensor(np.asarray(tr) + base[d], device=dev)])
            ho_y.append(yd[torch.as_tensor(np.asarray(ho) + base[d], device=dev)])
            lam_rows.append(d)
            owner.append(d)
    p_of = [int(np.asarray(X).shape[1]) for X, _ in data]
    train = _problem_set(Xd, tr_y, tr_rows, P, 1)
    held = _problem_set(Xd, ho_y, ho_rows, P, 1)
    pq = torch.as_tensor(np.array([p_of[d] for d in owner], np.int32), device=dev)
    train.p, held.p = pq, pq
    lam = path[torch.as_tensor(np.array(lam_rows, np.int64), device=dev)].contiguous()
    out = ll.fit(train, lam, opts=opts)
    loss = ll.path_loss(held, out["b"])
    lam_h = path.cpu().numpy()
    loss_h = loss.cpu().numpy()
    b_h = out["b"].cpu().numpy()
    st_h = out["status"].cpu().numpy()
    res = []
    s0 = 0
    for d, sp in enumerate(splits):
        S = len(sp)
        sl = slice(s0, s0 + S)
        nho = np.array([len(ho) for _, ho in sp], np.float64)
        per_row = loss_h[sl] / np.maximum(nho, 1)[:, None]
        mean = per_row.mean(axis=0)
        res.append(CVResult(lambdas=lam_h[d], loss=loss_h[sl], mean_loss=mean,
                            best=int(np.argmin(mean)), b=b_h[sl, :, :p_of[d]],
                            status=st_h[sl]))
        s0 += S
    return res


def cross_validate(X, y, K: int = 5, L: int = 16, ratio: float = 1e-3, seed: int = 0,
                   opts: ll.Opts | None = None, device="cuda") -> CVResult:
    """K-fold cross-validation of lambda for one data set."""
    n = np.asarray(X).shape[0]
    return cross_validate_many([(X, y)], [kfold_splits(n, K, seed)], L, ratio, opts, device)[0]

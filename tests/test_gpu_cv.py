"""Held-out loss kernel and the cross-validation driver on the GPU."""
import numpy as np
import pytest

import oracle
from paper_2510_15649_gb300 import synth

from gpu_common import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ll():
    import torch  # noqa: F401
    from paper_2510_15649_gb300 import build
    build.build()
    from paper_2510_15649_gb300 import ladlasso
    return ladlasso


def test_path_loss_matches_the_definition(ll):
    import torch
    batch = synth.batched_like(40, 0, 700, 1, 12, R=800, P=12, seed=51)
    pr = ll.Problems.from_numpy(batch)
    L = 3
    rng = np.random.default_rng(2)
    b = rng.standard_normal((40, L, 12)).astype(np.float32)
    for q in range(40):
        b[q, :, batch["p"][q]:] = 0.0
    loss = ll.path_loss(pr, torch.as_tensor(b, device="cuda")).cpu().numpy()
    for q in range(40):
        X, y = oracle.problem(batch, q)
        for l in range(L):
            ref = np.sum(np.abs(y - X @ b[q, l, :X.shape[1]].astype(np.float64)))
            assert abs(loss[q, l] - ref) <= 2e-5 * max(1.0, ref), (q, l, loss[q, l], ref)


def test_path_loss_bad_rows_give_nan(ll):
    import torch
    batch = synth.batched_like(3, 10, 50, 2, 4, R=60, P=4, seed=52)
    ri = batch["row_idx"].copy()
    ri[batch["offsets"][1]] = 10_000
    batch["row_idx"] = ri
    pr = ll.Problems.from_numpy(batch)
    loss = ll.path_loss(pr, torch.zeros((3, 2, 4), device="cuda")).cpu().numpy()
    assert np.all(np.isnan(loss[1])) and np.all(np.isfinite(loss[[0, 2]]))


def test_cross_validation_driver(ll):
    from paper_2510_15649_gb300 import cv
    rng = np.random.default_rng(5)
    n, p = 300, 8
    X = rng.standard_normal((n, p)).astype(np.float32)
    bt = np.zeros(p)
    bt[[1, 4]] = [2.0, -1.5]
    y = (X @ bt + rng.laplace(0, 1, n)).astype(np.float32)
    res = cv.cross_validate(X, y, K=4, L=8, ratio=1e-3, seed=0)
    sp = cv.kfold_splits(n, 4, 0)
    # held-out losses equal the definition at the returned coefficients
    for k, (tr, ho) in enumerate(sp):
        for l in range(8):
            ref = np.sum(np.abs(y[ho].astype(np.float64) - X[ho].astype(np.float64) @ res.b[k, l].astype(np.float64)))
            assert abs(res.loss[k, l] - ref) <= 2e-5 * max(1.0, ref)
    # the fits are the oracle's on the training rows
    batch = dict(X=X, y=np.concatenate([y[tr] for tr, _ in sp]),
                 row_idx=np.concatenate([tr for tr, _ in sp]).astype(np.int32),
                 offsets=np.concatenate([[0], np.cumsum([len(tr) for tr, _ in sp])]).astype(np.int64),
                 p=np.full(4, p, np.int32))
    lam = np.tile(res.lambdas.astype(np.float32), (4, 1))
    bfull = np.zeros((4, 8, p), np.float32)
    bfull[:] = res.b
    objs = np.array([[oracle.objective(*oracle.problem(batch, k), res.b[k, l].astype(np.float64), lam[k, l])
                      for l in range(8)] for k in range(4)], np.float32)
    out = compare(batch, lam, bfull, objs, res.status, problems=[0, 3])
    assert not out["bad"], out["bad"][:5]
    assert res.best == int(np.argmin(res.mean_loss))
    # the planted model: the chosen lambda keeps both true coefficients
    assert np.all(res.b[:, res.best, [1, 4]] != 0)


def test_cross_validate_many_matches_single(ll):
    from paper_2510_15649_gb300 import cv
    rng = np.random.default_rng(6)
    data = []
    for n, p in [(120, 3), (200, 6)]:
        X = rng.standard_normal((n, p)).astype(np.float32)
        y = (X[:, 0] * 1.5 + rng.laplace(0, 1, n)).astype(np.float32)
        data.append((X, y))
    many = cv.cross_validate_many(data, [cv.kfold_splits(len(y), 3, 1) for _, y in data], L=5)
    for (X, y), r in zip(data, many):
        one = cv.cross_validate(X, y, K=3, L=5, seed=1)
        np.testing.assert_allclose(r.lambdas, one.lambdas, rtol=1e-6)
        np.testing.assert_allclose(r.loss, one.loss, rtol=1e-4)
        assert r.b.shape == one.b.shape

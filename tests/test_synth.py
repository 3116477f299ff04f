"""The seeded input recipes: sizes, ranges, structure and determinism of
every workload generator (tiny, batched, large, diff, serving trace)."""
import numpy as np
import pytest

from paper_2510_15649_gb300 import synth


def _same(a, b):
    return all(np.array_equal(a[k], b[k]) for k in a if isinstance(a[k], np.ndarray))


def test_tiny_recipe():
    t = synth.tiny()
    assert t["X"].shape == (40, 4) and t["y"].shape == (40,) and t["X"].dtype == np.float32
    assert np.array_equal(t["b_true"], [1.5, 0.0, -2.0, 0.0]) and t["lam"] == 2.0
    # four rows carry the +10 shift; Laplace(0, 0.5) noise stays far below 5 at n = 40
    r = t["y"] - t["X"].astype(np.float64) @ t["b_true"]
    assert np.sum(r > 5.0) == 4 and np.all(np.abs(r[r <= 5.0]) < 5.0)
    assert _same(t, synth.tiny())


def test_batched_recipe():
    b = synth.batched()
    B = 4096
    n = np.diff(b["offsets"])
    assert b["X"].shape == (2000, 32) and len(n) == B and len(b["p"]) == B
    assert n.min() >= 50 and n.max() <= 2000 and b["p"].min() >= 4 and b["p"].max() <= 32
    assert b["offsets"][0] == 0 and b["offsets"][-1] == len(b["y"]) == len(b["row_idx"])
    # n ~ U{50..2000}: mean 1025 (sd of the mean 563 / 64 = 8.8)
    assert abs(n.mean() - 1025.0) < 45.0
    # p ~ U{4..32}: mean 18 (sd of the mean 8.4 / 64 = 0.13)
    assert abs(b["p"].mean() - 18.0) < 0.7
    for q in (0, 1, 2047, 4095):
        r = b["row_idx"][b["offsets"][q]:b["offsets"][q + 1]]
        assert np.all(np.diff(r) > 0) and r[0] >= 0 and r[-1] < 2000  # sorted, no repeats
    assert _same(b, synth.batched())
    assert not np.array_equal(b["y"][:50], synth.batched(B=8, seed=2)["y"][:50])


def test_batched_targets_follow_a_three_sparse_model():
    # y = X_b b_true + t(2) noise with 3 nonzeros: a regression of a long
    # problem on its p columns shows three large coefficients
    b = synth.batched_like(4, 1500, 2000, 10, 10, seed=7)
    for q in range(4):
        o0, o1 = b["offsets"][q], b["offsets"][q + 1]
        X = b["X"][b["row_idx"][o0:o1], :10].astype(np.float64)
        y = b["y"][o0:o1].astype(np.float64)
        coef = np.linalg.lstsq(X, y, rcond=None)[0]
        # least squares under t(2) noise is noisy, but at n >= 1500 the 7
        # zero coefficients stay below 0.5 and most of the 3 true ones
        # (U(-3, 3)) rise above it
        assert 2 <= np.sum(np.abs(coef) > 0.5) <= 3


def test_large_recipe_on_a_small_instance():
    L = synth.large(B=2, n=4000, p=16)
    assert L["X"].shape == (8000, 16) and L["row_idx"] is None
    assert np.array_equal(L["offsets"], [0, 4000, 8000]) and np.all(L["p"] == 16)
    X = L["X"].astype(np.float64)
    # AR(1) across columns with rho = 0.5: unit variance, lag-1 correlation 0.5, lag-2 0.25
    assert np.all(np.abs(X.var(axis=0) - 1.0) < 0.1)
    c1 = np.mean([np.corrcoef(X[:, j], X[:, j + 1])[0, 1] for j in range(15)])
    c2 = np.mean([np.corrcoef(X[:, j], X[:, j + 2])[0, 1] for j in range(14)])
    assert abs(c1 - 0.5) < 0.03 and abs(c2 - 0.25) < 0.03
    assert _same(L, synth.large(B=2, n=4000, p=16))


def test_diff_recipe():
    d = synth.diff(B=6)
    tr, va = d["train"], d["val"]
    assert tr["X"].shape == (6 * 400, 16) and va["X"].shape == (6 * 100, 16)
    assert np.array_equal(tr["offsets"], np.arange(7) * 400)
    assert np.array_equal(va["offsets"], np.arange(7) * 100)
    assert np.all(tr["p"] == 16) and np.all(va["p"] == 16)


def test_serving_trace_recipe():
    tr = synth.serve_trace(rate=20000.0, seconds=0.25, seed=4)
    t = np.array([r["t"] for r in tr])
    n = np.array([r["X"].shape[0] for r in tr])
    p = np.array([r["X"].shape[1] for r in tr])
    # Poisson arrivals: ~5000 in 0.25 s (sd 71), increasing times
    assert abs(len(tr) - 5000) < 300 and np.all(np.diff(t) > 0) and t[-1] < 0.25
    assert n.min() >= 20 and n.max() <= 5000 and p.min() >= 2 and p.max() <= 64
    # log-uniform n on [20, 5000]: mean (5000 - 20) / ln 250 = 902
    assert abs(n.mean() - 902.0) < 60.0
    # log-uniform: the median is the geometric mean, sqrt(20 * 5000) = 316
    assert abs(np.median(n) - 316.0) < 30.0
    assert all(r["y"].shape == (r["X"].shape[0],) for r in tr[:50])
    again = synth.serve_trace(rate=20000.0, seconds=0.25, seed=4)
    assert len(again) == len(tr) and np.array_equal(again[7]["y"], tr[7]["y"])
    assert len(synth.serve_trace(rate=20000.0, seconds=0.25, seed=4, max_requests=10)) == 10
    # a shared row bank: views of one N(0,1) matrix, the same size mix,
    # each request's own targets (its coefficients, noise and outliers)
    bk = synth.serve_trace(rate=20000.0, seconds=0.05, seed=4, bank_rows=20000)
    nb = np.array([r["X"].shape[0] for r in bk])
    assert abs(len(bk) - 1000) < 130 and nb.min() >= 20 and nb.max() <= 5000
    base = bk[0]["X"].base
    assert base is not None and all(r["X"].base is base for r in bk)
    assert base.shape == (20000, 64) and abs(float(base.std()) - 1.0) < 0.01
    for r in bk[:20]:
        X = r["X"].astype(np.float64)
        res = r["y"] - X @ np.linalg.lstsq(X, r["y"], rcond=None)[0]
        assert r["X"].dtype == np.float32 and r["y"].shape == (X.shape[0],)
        assert np.abs(res).max() > 0  # noise on every request
    with pytest.raises(ValueError):
        synth.serve_trace(rate=100.0, seconds=0.1, seed=1, bank_rows=100)

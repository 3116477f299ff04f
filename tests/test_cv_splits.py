"""Host logic of the cross-validation driver: the splits it builds, and what
it hands the library for each split (rows, lambda path, columns) and how it
reduces the held-out losses to the chosen lambda."""
import numpy as np

from paper_2510_15649_gb300.cv import kfold_splits, subset_splits


def test_kfold_partitions_the_rows():
    sp = kfold_splits(103, 5, seed=3)
    assert len(sp) == 5
    held = np.concatenate([ho for _, ho in sp])
    assert np.array_equal(np.sort(held), np.arange(103))
    for tr, ho in sp:
        assert len(np.intersect1d(tr, ho)) == 0
        assert np.array_equal(np.union1d(tr, ho), np.arange(103))
        assert np.all(np.diff(tr) > 0) and np.all(np.diff(ho) > 0)
        assert abs(len(ho) - 103 / 5) < 1


def test_split_arguments_are_checked():
    import pytest
    for n, K in [(10, 1), (10, 11), (0, 2)]:
        with pytest.raises(ValueError):
            kfold_splits(n, K)
    for n, m, S in [(10, 0, 3), (10, 10, 3), (10, 3, 0)]:
        with pytest.raises(ValueError):
            subset_splits(n, m, S)
    assert len(kfold_splits(10, 10)) == 10  # leave-one-out


def test_subset_splits_hold_out_m_rows():
    sp = subset_splits(50, 7, 9, seed=1)
    assert len(sp) == 9
    for tr, ho in sp:
        assert len(ho) == 7 and len(tr) == 43
        assert len(np.intersect1d(tr, ho)) == 0
    assert len({tuple(ho) for _, ho in sp}) > 1


# ------------------------------------------------------------------ the
# driver's host logic on CPU tensors, with its four library calls replaced
# by a fake that records what it is given


class FakeLibrary:
    """lambda_max follows its definition; fit records the problem sets it
    gets and returns b = 0; path_loss returns, for problem k and path
    position l, sum over the problem's rows of |y| times (1 + (l - 2)^2),
    so the driver's normalisation and argmin can be checked."""

    def __init__(self):
        self.train = None
        self.held = None
        self.lam = None

    @staticmethod
    def rows_of(pr):
        off = pr.offsets.numpy()
        ri = pr.row_idx.numpy()
        return [ri[off[k]:off[k + 1]] for k in range(len(off) - 1)], \
               [pr.y.numpy()[off[k]:off[k + 1]] for k in range(len(off) - 1)]

    def lambda_max(self, pr, ws=None, stream=None):
        import torch
        off, p = pr.offsets.numpy(), pr.p.numpy()
        X, y = pr.X.numpy(), pr.y.numpy()
        return torch.tensor([np.abs(X[off[q]:off[q + 1], :p[q]].T @ np.sign(y[off[q]:off[q + 1]])).max()
                             for q in range(len(off) - 1)], dtype=torch.float32)

    def lambda_path(self, lmax, L, ratio=1e-3, stream=None):
        import torch
        t = np.arange(L) / max(1, L - 1)
        return torch.from_numpy((lmax.numpy()[:, None] * ratio ** t).astype(np.float32))

    def fit(self, pr, lambdas, *, opts=None, **kw):
        import torch
        self.train, self.lam = pr, lambdas.numpy().copy()
        B, L = self.lam.shape
        return dict(b=torch.zeros((B, L, pr.P)), obj=torch.zeros((B, L)),
                    status=torch.zeros((B, L), dtype=torch.int32))

    def path_loss(self, pr, b, stream=None):
        import torch
        self.held = pr
        _, ys = self.rows_of(pr)
        L = b.shape[1]
        w = 1.0 + (np.arange(L) - 2.0) ** 2
        return torch.from_numpy(np.array([np.abs(y).sum() * w for y in ys], np.float32))


def test_driver_hands_each_split_its_rows_path_and_columns(monkeypatch):
    from paper_2510_15649_gb300 import cv
    from paper_2510_15649_gb300 import ladlasso as ll
    f = FakeLibrary()
    for name in ("lambda_max", "lambda_path", "fit", "path_loss"):
        monkeypatch.setattr(ll, name, getattr(f, name))
    rng = np.random.default_rng(4)
    data = [(rng.standard_normal((40, 3)).astype(np.float32), rng.standard_normal(40).astype(np.float32)),
            (rng.standard_normal((55, 5)).astype(np.float32), rng.standard_normal(55).astype(np.float32))]
    splits = [cv.kfold_splits(40, 4, seed=1), cv.subset_splits(55, 6, 3, seed=2)]
    L = 6
    res = cv.cross_validate_many(data, splits, L=L, ratio=1e-2, device="cpu")
    assert len(res) == 2
    tr_rows, tr_y = f.rows_of(f.train)
    ho_rows, ho_y = f.rows_of(f.held)
    k = 0
    base = [0, 40]
    for d, ((X, y), sp) in enumerate(zip(data, splits)):
        lmax = np.abs(X.T @ np.sign(y)).max()
        path = lmax * 1e-2 ** (np.arange(L) / (L - 1))
        np.testing.assert_allclose(res[d].lambdas, path, rtol=1e-5)
        for s, (tr, ho) in enumerate(sp):
            # each split: its training rows of its own data set, in the stacked design
            assert np.array_equal(tr_rows[k], tr + base[d])
            assert np.array_equal(ho_rows[k], ho + base[d])
            assert np.array_equal(tr_y[k], y[tr]) and np.array_equal(ho_y[k], y[ho])
            assert f.train.p.numpy()[k] == X.shape[1] and f.held.p.numpy()[k] == X.shape[1]
            np.testing.assert_allclose(f.lam[k], path, rtol=1e-5)
            k += 1
        # the stacked design holds the data set's columns, zero-padded
        Xd = f.train.X.numpy()[base[d]:base[d] + X.shape[0]]
        assert np.array_equal(Xd[:, :X.shape[1]], X) and np.all(Xd[:, X.shape[1]:] == 0)
        # mean over splits of the per-row held-out loss; argmin at position 2
        w = 1.0 + (np.arange(L) - 2.0) ** 2
        want = np.mean([np.abs(y[ho]).sum() / len(ho) for _, ho in sp]) * w
        np.testing.assert_allclose(res[d].mean_loss, want, rtol=1e-5)
        assert res[d].best == 2 and res[d].best_lambda == res[d].lambdas[2]
        assert res[d].b.shape == (len(sp), L, X.shape[1])
    assert k == len(tr_rows) == len(ho_rows) == 7

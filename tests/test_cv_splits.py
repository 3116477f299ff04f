"""Host logic of the cross-validation driver: the splits it builds."""
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


def test_subset_splits_hold_out_m_rows():
    sp = subset_splits(50, 7, 9, seed=1)
    assert len(sp) == 9
    for tr, ho in sp:
        assert len(ho) == 7 and len(tr) == 43
        assert len(np.intersect1d(tr, ho)) == 0
    assert len({tuple(ho) for _, ho in sp}) > 1

"""Host logic of the server: the problem set that computes lambda_max for
newly admitted slots must pass the library's offset rule (non-negative,
non-decreasing, last offset equal to the pool's row count) while each
problem still starts at its own slot and has room for a full slot."""
import numpy as np
import pytest

from paper_2510_15649_gb300.serve import admission_offsets


def _library_accepts(offsets, total_rows):
    # the rule ladlasso_lambda_max / ladlasso_fit_batched apply to offsets
    o = np.asarray(offsets, np.int64)
    return bool(np.all(o >= 0) and np.all(o <= total_rows) and np.all(np.diff(o) >= 0)
                and o[-1] == total_rows)


@pytest.mark.parametrize("slots", [[0], [0, 1, 2], [3], [1, 5, 6], [7], [0, 7], [2, 4, 6, 7]])
def test_admission_offsets_pass_the_library_rule(slots):
    S, cap = 8, 300
    off = admission_offsets(np.array(slots), cap, S)
    assert len(off) == len(slots) + 1
    assert _library_accepts(off, S * cap)
    assert np.array_equal(off[:-1], np.array(slots) * cap)
    assert np.all(np.diff(off) >= cap)


def test_offsets_ending_at_the_last_new_slot_were_rejected():
    # the form that ended the set at (last new slot + 1) * cap fails the
    # rule whenever the last slot of the pool is not among the new ones
    S, cap, ss = 8, 300, np.array([0, 2])
    assert not _library_accepts(np.append(ss * cap, (ss[-1] + 1) * cap), S * cap)

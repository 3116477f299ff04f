"""Host helpers of bench.py: the clock summary that accepts or rejects a
run, and the row-update and shared-memory byte counts behind the
roofline."""
import importlib.util
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_clock_summary():
    b = _bench()
    cs = b.ClockSampler()
    assert cs.summary()["reasons"] == ["unsampled"]
    idle = ["Not Active"] * 4
    cs.rows = [["2070", "2070", "900.1"] + idle,
               ["1980", "2070", "1200.0", "Not Active", "Not Active", "Not Active", "Active"],
               ["2040", "2070", "1100.0"] + idle,
               ["[N/A]", "2070", "[N/A]"] + idle]
    s = cs.summary()
    assert s["sm_mhz"] == 2040.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 4
    assert s["reasons"] == ["sw_power_cap"]
    cs.rows.append(["1500", "2070", "1300", "Active", "Not Active", "Active", "Not Active"])
    assert cs.summary()["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_row_updates_and_smem_bytes():
    b = _bench()
    batch = dict(offsets=np.array([0, 10, 30], np.int64), p=np.array([3, 5], np.int32))
    cnt = np.zeros((2, 2, 8), np.int32)
    cnt[0, :, 4] = [6, 2]   # selection passes of problem 0 at its two path positions
    cnt[1, :, 4] = [1, 9]
    cnt[0, :, 5] = [4, 2]   # 1-D steps
    cnt[1, :, 5] = [1, 7]
    # n x steps per fit
    assert b.row_updates(batch, cnt, 2) == (4 + 2) * 10 + (1 + 7) * 20
    # n x (8 B per pass + 12 B per step) per fit
    want = (8 * 6 + 12 * 4) * 10 + (8 * 2 + 12 * 2) * 10 + (8 * 1 + 12 * 1) * 20 + (8 * 9 + 12 * 7) * 20
    assert b.smem_bytes(batch, cnt, 2) == want
    # one pass per step: 20 B per row-update
    one = np.zeros((1, 1, 8), np.int32)
    one[0, 0, 4] = one[0, 0, 5] = 3
    b1 = dict(offsets=np.array([0, 7], np.int64), p=np.array([2], np.int32))
    assert b.smem_bytes(b1, one, 1) == 20 * b.row_updates(b1, one, 1)


def test_log2_histogram():
    b = _bench()
    h = b.log2_histogram(np.array([0, 1, 2, 3, 4, 7, 8, 15, 16, 1000]))
    assert h["lower_edges"] == [0, 1, 2, 4, 8, 16, 32, 64, 128, 256, 512]
    assert h["counts"] == [1, 1, 2, 2, 2, 1, 0, 0, 0, 0, 1]
    assert sum(h["counts"]) == 10
    assert b.log2_histogram(np.zeros(3, np.int32)) == {"lower_edges": [0], "counts": [3]}

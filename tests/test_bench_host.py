"""Host helpers of bench.py: the clock summary that accepts or rejects a
run, the rule that reports ncu traffic only for the kernel code and launch
shape it was captured on, and the row-update count behind the roofline."""
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


def test_traffic_only_for_the_captured_code_and_shape():
    b = _bench()
    name = "launches_batched4096.md"
    src = "paper_2510_15649_gb300/csrc/fit_block.cu"
    text = open(os.path.join(ROOT, "profiles", name)).read()
    assert "kernel_code_sha256:" in text and "traffic_bytes_per_launch[" in text
    # another source file never matches the recorded code hash
    assert b.profile_traffic(name, "paper_2510_15649_gb300/csrc/aux_kernels.cu", "32x3/o0") is None
    # no launch shape, or one that was not captured
    assert b.profile_traffic(name, src, None) is None
    assert b.profile_traffic(name, src, "32x99/o1") is None
    # a missing profile
    assert b.profile_traffic("no_such_profile.md", src, "32x3/o0") is None
    # a captured shape gives the recorded number, or None once the code has changed
    v = b.profile_traffic(name, src, "32x3/o0")
    assert v is None or (v > 0 and f"traffic_bytes_per_launch[32x3/o0]:" in text)


def test_row_updates_count():
    b = _bench()
    batch = dict(offsets=np.array([0, 10, 30], np.int64), p=np.array([3, 5], np.int32))
    cnt = np.zeros((2, 2, 8), np.int32)
    cnt[0, :, 0] = [4, 2]   # sweeps of problem 0 at its two path positions
    cnt[1, :, 0] = [1, 3]
    cnt[0, :, 2] = [0, 7]   # polish pivots
    cnt[1, :, 2] = [5, 0]
    # (sweeps * p + pivots) * n per fit
    want = (4 * 3 + 0) * 10 + (2 * 3 + 7) * 10 + (1 * 5 + 5) * 20 + (3 * 5 + 0) * 20
    assert b.row_updates(batch, cnt, 2) == want


def test_log2_histogram():
    b = _bench()
    h = b.log2_histogram(np.array([0, 1, 2, 3, 4, 7, 8, 15, 16, 1000]))
    assert h["lower_edges"] == [0, 1, 2, 4, 8, 16, 32, 64, 128, 256, 512]
    assert h["counts"] == [1, 1, 2, 2, 2, 1, 0, 0, 0, 0, 1]
    assert sum(h["counts"]) == 10
    assert b.log2_histogram(np.zeros(3, np.int32)) == {"lower_edges": [0], "counts": [3]}

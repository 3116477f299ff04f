"""The GPU parity harness itself (tests/gpu_common.py), on the CPU: fed the
oracle's own results as the kernel's output it reports nothing, and each
kind of error it exists to catch, planted in that output, is reported.  A
harness that passed everything would make the GPU parity tests vacuous."""
import numpy as np
import pytest

import oracle
from gpu_common import compare, compare_parallel
from paper_2510_15649_gb300 import synth

L = 3


@pytest.fixture(scope="module")
def case():
    batch = synth.batched_like(6, 30, 120, 2, 6, R=150, P=6, seed=19)
    B = 6
    lam = np.zeros((B, L), np.float32)
    b = np.zeros((B, L, 6), np.float32)
    obj = np.zeros((B, L), np.float32)
    st = np.zeros((B, L), np.int32)
    for q in range(B):
        X, y = oracle.problem(batch, q)
        lam[q] = (oracle.lambda_max(X, y) * np.array([0.5, 0.1, 0.01])).astype(np.float32)
        r = oracle.fit_path(X, y, lam[q].astype(np.float64))
        p = X.shape[1]
        b[q, :, :p] = r["b"]
        for l in range(L):
            obj[q, l] = oracle.objective(X, y, b[q, l, :p].astype(np.float64), float(lam[q, l]))
        st[q] = r["status"]
    return batch, lam, b, obj, st


def _kinds(res):
    return {x[2] for x in res["bad"]}


def test_the_oracles_own_results_pass(case):
    batch, lam, b, obj, st = case
    res = compare(batch, lam, b, obj, st)
    assert res["checked"] == 6 * L and not res["bad"], res["bad"]


def test_planted_errors_are_reported(case):
    batch, lam, b, obj, st = case
    p0 = int(batch["p"][0])
    # a coefficient moved far enough to raise the objective
    bb = b.copy()
    bb[0, 1, 0] += 0.5
    assert "obj" in _kinds(compare(batch, lam, bb, obj, st, problems=[0]))
    # a tiny move: objective within tolerance, coefficient error reported
    # where the optimum is unique
    bb = b.copy()
    q, l = next((q, l) for q in range(6) for l in range(L)
                if st[q, l] == 0 and np.any(b[q, l] != 0))
    j = int(np.flatnonzero(b[q, l])[0])
    bb[q, l, j] *= 1.0 + 1e-3
    kinds = _kinds(compare(batch, lam, bb, obj, st, problems=[q]))
    assert kinds & {"coef", "obj"}, kinds
    # a support entry zeroed
    bb = b.copy()
    bb[q, l, j] = 0.0
    assert _kinds(compare(batch, lam, bb, obj, st, problems=[q])) & {"support", "obj"}
    # obj_out that does not match the returned coefficients
    oo = obj.copy()
    oo[1, 0] *= 1.01
    assert "obj_out" in _kinds(compare(batch, lam, b, oo, st, problems=[1]))
    # nonzero padding beyond p
    assert p0 < 6
    bb = b.copy()
    bb[0, 0, p0] = 1.0
    assert "padding" in _kinds(compare(batch, lam, bb, obj, st, problems=[0]))
    # bad input that the kernel did not report
    lb = lam.copy()
    lb[2, 1] = np.nan
    assert "status" in _kinds(compare(batch, lb, b, obj, st, problems=[2]))


def test_parallel_form_reports_the_same(case):
    batch, lam, b, obj, st = case
    bb = b.copy()
    bb[4, 2, 0] += 0.5
    one = compare(batch, lam, bb, obj, st)
    par = compare_parallel(batch, lam, bb, obj, st, range(6), workers=3)
    assert par["checked"] == one["checked"]
    assert sorted(map(str, par["bad"])) == sorted(map(str, one["bad"]))

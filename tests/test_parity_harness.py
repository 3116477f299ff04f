"""The GPU parity harness itself (tests/gpu_common.py), on the CPU: fed the
oracle's own results as the kernel's output it reports nothing, and each
kind of error it exists to catch, planted in that output, is reported.  A
harness that passed everything would make the GPU parity tests vacuous."""
import numpy as np
import pytest

import oracle
from gpu_common import EXACT_CHOP_OPTS, compare, compare_parallel, exact_problems
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


def test_gradient_check_accepts_the_oracle_and_rejects_planted_errors():
    from test_gpu_backward import _check_against_oracle
    d = synth.diff(B=6, n=140, n_train=110, p=6, seed=3)
    tr, va = d["train"], d["val"]
    B, P = 6, 6
    lam = np.array([0.1 * oracle.lambda_max(*oracle.problem(tr, q)) for q in range(B)], np.float32)
    up = np.linspace(0.5, 2.0, B)
    g = dict(y=np.zeros(len(tr["y"])), X=np.zeros((len(tr["y"]), P)), yv=np.zeros(len(va["y"])),
             Xv=np.zeros((len(va["y"]), P)), lam=np.zeros(B), status=np.zeros(B, np.int32),
             loss=np.zeros(B))
    bg = np.zeros((B, P), np.float32)
    for q in range(B):
        X, y = oracle.problem(tr, q)
        Xv, yv = oracle.problem(va, q)
        r = oracle.fit_path(X, y, [float(lam[q])])
        bg[q] = r["b"][0]
        og = oracle.grad(X, y, r["b"][0], r["basis"][0], Xv, yv, up=float(up[q]))
        o0, o1 = tr["offsets"][q], tr["offsets"][q + 1]
        v0, v1 = va["offsets"][q], va["offsets"][q + 1]
        g["y"][o0:o1], g["X"][o0:o1] = og["gy"], og["gX"]
        g["yv"][v0:v1], g["Xv"][v0:v1] = og["gyv"], og["gXv"]
        g["loss"][q] = np.abs(yv - Xv @ r["b"][0]).sum()
        g["status"][q] = 0 if og["ok"] else 4
    assert _check_against_oracle(g, bg, lam, up, tr, va, range(B)) >= B // 2
    for key, idx, delta in [("y", None, 0.1), ("Xv", None, 0.1), ("loss", 0, 1.0), ("lam", 0, 0.5)]:
        bad = {k: v.copy() for k, v in g.items()}
        if idx is None:  # a gradient entry of a checked problem's rows
            o0 = tr["offsets"][0] if key == "y" else va["offsets"][0]
            nz = np.flatnonzero(np.atleast_2d(bad[key].T)[0][o0:] != 0)
            pos = o0 + (nz[0] if len(nz) else 0)
            bad[key][pos] += delta
        else:
            bad[key][idx] += delta
        with pytest.raises(AssertionError):
            _check_against_oracle(bad, bg, lam, up, tr, va, range(B))


def test_vertex_from_basis_codes_reproduces_the_oracle():
    # the large-workload test rebuilds the FP64 vertex of a reported basis
    # (row codes i >= 0, coordinate codes -(j+1)); on the oracle's own basis
    # it must give the oracle's vertex
    from test_gpu_large import _vertex
    rng = np.random.default_rng(5)
    checked = 0
    for n, p in [(40, 3), (120, 8)]:
        X = rng.standard_normal((n, p))
        y = X @ np.where(rng.random(p) < 0.5, rng.uniform(-2, 2, p), 0.0) + rng.laplace(0, 0.5, n)
        for frac in (0.5, 0.05):
            lam = frac * oracle.lambda_max(X, y)
            r = oracle.fit_path(X, y, [lam])
            if r["status"][0] != oracle.FIT_OK:
                continue
            np.testing.assert_allclose(_vertex(X, y, r["basis"][0]), r["b"][0], atol=1e-9)
            checked += 1
    assert checked >= 2


def test_vertex_multiplier_check_agrees_with_the_oracle_certificate():
    # the large-workload test falls back on the vertex's own multipliers
    # where the oracle's certificate takes a row within its zero threshold
    # for one on its hyperplane; away from that case the two must agree:
    # True at the oracle's optimal bases, False at other vertices
    from test_gpu_large import _kkt_at_vertex, _vertex
    rng = np.random.default_rng(11)
    seen = {True: 0, False: 0}
    for n, p in [(60, 3), (150, 6)]:
        X = rng.standard_normal((n, p))
        y = X @ np.where(rng.random(p) < 0.5, rng.uniform(-2, 2, p), 0.0) + rng.laplace(0, 0.5, n)
        for frac in (0.5, 0.1, 0.01):
            lam = frac * oracle.lambda_max(X, y)
            r = oracle.fit_path(X, y, [lam])
            cands = [r["basis"][0]] if r["status"][0] == oracle.FIT_OK else []
            for _ in range(12):
                k = rng.integers(0, p + 1)
                rows = rng.choice(n, k, replace=False)
                cols = rng.choice(p, p - k, replace=False)
                cands.append(np.concatenate([rows, -(cols + 1)]).astype(np.int32))
            for codes in cands:
                try:
                    bv = _vertex(X, y, codes)
                except np.linalg.LinAlgError:
                    continue
                res = y - X @ bv
                off = np.ones(n, bool)
                off[codes[codes >= 0]] = False
                if np.any(np.abs(res[off]) <= 1e-6 * max(1.0, np.abs(y).max())):
                    continue  # a row on (or near) its hyperplane: degenerate
                F = oracle.objective(X, y, bv, lam)
                gap, _ = oracle.certify(X, y, bv, lam)
                want = bool(gap <= 1e-7 * max(1.0, F))
                assert _kkt_at_vertex(X, y, codes, lam) == want, (n, p, frac, codes)
                seen[want] += 1
    assert seen[True] >= 4 and seen[False] >= 20, seen


def test_exact_family_stays_exact_in_float32():
    # premise of the GPU test that compares chop-only fits bit for bit: on
    # these problems the oracle's results (and so every key, residual and
    # objective on the way, which have no more bits) are dyadic rationals
    # of at most 12 fractional bits below 2^8 in magnitude, objectives
    # below 2^12: all exact in float32's 24-bit significand
    probs, lam = exact_problems(73)
    o = oracle.default_opts(tol_move=1e-6, **EXACT_CHOP_OPTS)
    chopped = 0
    for (Xq, yq), lq in zip(probs, lam[:, 0]):
        X, y = Xq.astype(np.float64), yq.astype(np.float64)
        r = oracle.fit_path(X, y, [float(lq)], opts=o)
        b, f = r["b"][0], r["f"][0]
        assert np.all(b * 4096 == np.round(b * 4096)) and np.abs(b).max() < 256
        assert f * 4096 == round(f * 4096) and f < 4096
        assert np.array_equal(X.astype(np.float32).astype(np.float64), X)
        chopped += r["stats"][0]["chop_ran"]
    assert chopped >= len(probs) // 2

"""Pins for the FP64 oracle (CPU only).

Each test ties the oracle to something other than itself: the exact
vertex enumeration of Section 3.2 against the independent dense simplex of
Section 3.1 (and scipy's HiGHS LP), closed forms, invariances of the
objective, the duality-gap certificate and finite differences.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2510_15649_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def F(X, y, b, lam):
    return np.abs(y - X @ b).sum() + lam * np.abs(b).sum()


def rel(a, b):
    return abs(a - b) / max(1.0, abs(b))


def rand_problem(rng, n, p, outliers=True):
    X = rng.standard_normal((n, p))
    bt = np.zeros(p)
    k = min(2, p)
    bt[rng.choice(p, k, replace=False)] = rng.uniform(-3, 3, k)
    y = X @ bt + rng.laplace(0, 0.5, n)
    if outliers:
        y[rng.choice(n, max(1, n // 10), replace=False)] += 10
    return X, y


# ---------------------------------------------------------------- tiny

def test_tiny_golden_brute_simplex_method_agree():
    g = json.load(open(os.path.join(HERE, "golden", "tiny_fit.json")))
    t = synth.tiny()
    X, y, lam = t["X"].astype(float), t["y"].astype(float), float(t["lam"])
    fb, bb, nd = oracle.brute_force(X, y, lam)
    fs, bs = oracle.simplex(X, y, lam)
    r = oracle.fit_path(X, y, [lam])
    assert nd == 1
    assert rel(fb, g["F_star"]) < 1e-12
    assert rel(fs, fb) < 1e-12
    assert rel(r["f"][0], fb) < 1e-12
    assert np.max(np.abs(r["b"][0] - bb)) < 1e-9
    assert np.max(np.abs(bb - np.array(g["b_star"]))) < 1e-9
    assert r["status"][0] == oracle.FIT_OK
    gap, info = oracle.certify(X, y, r["b"][0], lam)
    assert gap < 1e-9 and info["unique"]


def test_golden_file_is_what_its_script_computes():
    # the stored expected values come only from tests/golden/make_golden.py,
    # which calls only oracle/: recomputing gives the stored file
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    fresh = mg.compute()
    stored = json.load(open(os.path.join(HERE, "golden", "tiny_fit.json")))
    assert set(fresh) == set(stored)
    for k, v in stored.items():
        if isinstance(v, float):
            assert rel(fresh[k], v) < 1e-12, k
        elif isinstance(v, list):
            np.testing.assert_allclose(fresh[k], v, rtol=1e-12, atol=1e-14)
        else:
            assert fresh[k] == v, k


def test_simplex_matches_scipy_highs():
    linprog = pytest.importorskip("scipy.optimize").linprog
    rng = np.random.default_rng(11)
    for n, p in [(12, 3), (30, 5), (60, 8)]:
        X, y = rand_problem(rng, n, p)
        for lam in [0.05, 1.0, 5.0]:
            fs, _ = oracle.simplex(X, y, lam)
            c = np.concatenate([lam * np.ones(2 * p), np.ones(2 * n)])
            A = np.hstack([X, -X, np.eye(n), -np.eye(n)])
            res = linprog(c, A_eq=A, b_eq=y, bounds=(0, None), method="highs")
            assert rel(fs, res.fun) < 1e-9, (n, p, lam, fs, res.fun)


def test_dual_lp_value_equals_the_method_optimum():
    # strong duality for the LP of Section 3.1 with lambda on |b|_1: the
    # optimum equals max y.u over |u_i| <= 1, |(X^T u)_j| <= lambda (the
    # bounded dual form), solved here by scipy's HiGHS, independently of
    # the oracle's simplex, brute force and certificate
    linprog = pytest.importorskip("scipy.optimize").linprog
    rng = np.random.default_rng(12)
    for n, p in [(15, 2), (40, 4), (80, 6)]:
        X, y = rand_problem(rng, n, p)
        for lam in [0.1, 2.0, 0.9 * oracle.lambda_max(X, y)]:
            r = oracle.fit_path(X, y, [lam])
            A = np.vstack([X.T, -X.T])
            dual = linprog(-y, A_ub=A, b_ub=lam * np.ones(2 * p), bounds=(-1, 1), method="highs")
            assert dual.status == 0
            assert rel(r["f"][0], -dual.fun) < 1e-9, (n, p, lam, r["f"][0], -dual.fun)
            # and the certificate's dual point is feasible with the same value
            gap, info = oracle.certify(X, y, r["b"][0], lam)
            assert abs(gap) <= 1e-8 * max(1.0, r["f"][0])
            assert rel(info["dual"], -dual.fun) < 1e-8


def test_method_optimum_equals_highs_dual_at_workload_sizes():
    # the oracle's method at the sizes the GPU runs (the batched workload's
    # problems across its range of n, up to 2000 x 32; the large recipe at
    # 1500 x 64; the differentiation recipe's 400 x 16 training rows) against
    # the bounded dual LP (Section 3.1, lambda on |b|_1) solved by scipy's
    # HiGHS -- an exact solver that shares nothing with the method
    linprog = pytest.importorskip("scipy.optimize").linprog
    from paper_2510_15649_gb300 import synth
    cases = []
    b = synth.batched(B=4096, seed=1)
    n = np.diff(b["offsets"])
    for q in np.argsort(n, kind="stable")[np.linspace(0, 4095, 6).round().astype(int)]:
        cases.append(oracle.problem(b, int(q)))
    big = synth.large(B=1, n=1500, p=64, seed=3)
    cases.append((big["X"].astype(np.float64), big["y"].astype(np.float64)))
    d = synth.diff(B=2, seed=3)["train"]
    cases.append(oracle.problem(d, 1))
    for X, y in cases:
        p = X.shape[1]
        lm = oracle.lambda_max(X, y)
        lams = lm * np.array([0.5, 0.1, 0.01, 0.001])
        r = oracle.fit_path(X, y, lams)
        A = np.vstack([X.T, -X.T])
        for l, lam in enumerate(lams):
            dual = linprog(-y, A_ub=A, b_ub=lam * np.ones(2 * p), bounds=(-1, 1), method="highs")
            assert dual.status == 0
            assert rel(r["f"][l], -dual.fun) < 1e-9, (X.shape, l, r["f"][l], -dual.fun)
            assert r["status"][l] & 1 == 0


@pytest.mark.parametrize("seed", range(6))
def test_random_tiny_brute_equals_simplex_equals_method(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(6, 15))
    p = int(rng.integers(1, 5))
    X, y = rand_problem(rng, n, p)
    lmax = oracle.lambda_max(X, y)
    for lam in [0.9 * lmax, 0.2 * lmax, 0.02 * lmax, 1e-3 * lmax]:
        fb, bb, nd = oracle.brute_force(X, y, lam)
        fs, bs = oracle.simplex(X, y, lam)
        r = oracle.fit_path(X, y, [lam])
        assert rel(fs, fb) < 1e-11
        assert rel(r["f"][0], fb) < 1e-11, (n, p, lam)
        assert rel(F(X, y, r["b"][0], lam), fb) < 1e-11
        if nd == 1:
            assert np.max(np.abs(r["b"][0] - bb)) < 1e-7


def test_lambda_path_warm_start_matches_cold_fits():
    rng = np.random.default_rng(5)
    X, y = rand_problem(rng, 60, 6)
    lmax = oracle.lambda_max(X, y)
    lams = lmax * np.logspace(0, -3, 8)
    path = oracle.fit_path(X, y, lams)
    for l, lam in enumerate(lams):
        fs, _ = oracle.simplex(X, y, lam)
        assert rel(path["f"][l], fs) < 1e-11
        cold = oracle.fit_path(X, y, [lam])
        assert rel(cold["f"][0], fs) < 1e-11


def test_medium_method_equals_simplex_and_certificate():
    rng = np.random.default_rng(7)
    for n, p in [(200, 8), (400, 16)]:
        X, y = rand_problem(rng, n, p)
        lmax = oracle.lambda_max(X, y)
        lams = lmax * np.logspace(-0.3, -3, 4)
        path = oracle.fit_path(X, y, lams)
        for l, lam in enumerate(lams):
            fs, _ = oracle.simplex(X, y, lam)
            assert rel(path["f"][l], fs) < 1e-10, (n, p, lam)
            gap, info = oracle.certify(X, y, path["b"][l], lam)
            assert gap <= 1e-9 * max(1, path["f"][l])
            assert path["status"][l] in (oracle.FIT_OK, oracle.FIT_NONUNIQUE)


# ---------------------------------------------------------------- axis update

def test_axis_update_is_exact_1d_minimum():
    rng = np.random.default_rng(3)
    for trial in range(20):
        n, p = int(rng.integers(3, 30)), int(rng.integers(1, 5))
        X, y = rand_problem(rng, n, p)
        b = rng.standard_normal(p)
        lam = float(rng.uniform(0, 3))
        j = int(rng.integers(p))
        b1, r1, piv = oracle.axis_update(X, y, b, lam, j)
        # brute force over the 1-D breakpoints of the axis function
        r0 = y - X @ b
        nz = X[:, j] != 0
        cands = np.concatenate([b[j] + r0[nz] / X[nz, j], [0.0]])
        best = np.inf
        for t in cands:
            bt = b.copy()
            bt[j] = t
            best = min(best, F(X, y, bt, lam))
        assert F(X, y, b1, lam) <= best * (1 + 1e-13) + 1e-13
        assert np.all(np.delete(b1, j) == np.delete(b, j))
        np.testing.assert_allclose(r1, y - X @ b1, atol=1e-10)
        if piv >= 0:
            assert abs(r1[piv]) < 1e-9
        if piv == -1:
            assert b1[j] == 0.0


def test_p1_closed_form_weighted_median():
    # p = 1: argmin sum |y_i - x_i b| + lam |b| is the weighted median of
    # y_i / x_i (weights |x_i|) and 0 (weight lam) -- sorted by hand here.
    rng = np.random.default_rng(9)
    for trial in range(10):
        n = int(rng.integers(5, 40))
        x = rng.standard_normal((n, 1))
        y = 2 * x[:, 0] + rng.standard_normal(n)
        lam = float(rng.uniform(0, 2))
        z = np.concatenate([y / x[:, 0], [0.0]])
        w = np.concatenate([np.abs(x[:, 0]), [lam]])
        o = np.argsort(z)
        c = np.cumsum(w[o])
        k = np.searchsorted(c, c[-1] / 2)
        expect = z[o][k]
        r = oracle.fit_path(x, y, [lam])
        assert abs(r["b"][0, 0] - expect) < 1e-12 * max(1, abs(expect))


def test_flat_segment_tie_rule_keeps_current_value():
    # two rows y = 1 and y = 3 with x = 1, lam = 0: every b in [1, 3] is
    # optimal (a flat minimum, Section 3.5).  The axis update keeps a current
    # value inside the segment and moves an outside one to the nearer end.
    X = np.ones((2, 1))
    y = np.array([1.0, 3.0])
    for b0, expect in [(2.5, 2.5), (0.0, 1.0), (7.0, 3.0)]:
        b1, _, _ = oracle.axis_update(X, y, np.array([b0]), 0.0, 0)
        assert b1[0] == expect


# ---------------------------------------------------------------- special cases

def test_lambda_max_gives_zero_and_below_does_not():
    rng = np.random.default_rng(4)
    for trial in range(5):
        X, y = rand_problem(rng, 50, 6)
        lmax = oracle.lambda_max(X, y)
        assert abs(lmax - np.abs(X.T @ np.sign(y)).max()) < 1e-12 * lmax
        r = oracle.fit_path(X, y, [lmax * 1.0001, lmax * 5])
        assert np.all(r["b"] == 0.0)
        fs, bs = oracle.simplex(X, y, lmax * 0.95)
        assert fs < F(X, y, np.zeros(6), lmax * 0.95) - 1e-9
        r2 = oracle.fit_path(X, y, [lmax * 0.95])
        assert np.any(r2["b"][0] != 0.0)


def test_square_system_tiny_lambda_interpolates():
    rng = np.random.default_rng(8)
    for p in [1, 2, 3, 5]:
        X = rng.standard_normal((p, p)) + 3 * np.eye(p)
        y = rng.standard_normal(p) * 3
        lam = 1e-6
        b = np.linalg.solve(X, y)
        r = oracle.fit_path(X, y, [lam])
        # with lam small relative to the rows, the fit interpolates: b = X^-1 y
        if np.all(np.abs(np.linalg.solve(X.T, lam * np.sign(b))) < 1):
            np.testing.assert_allclose(r["b"][0], b, rtol=1e-9, atol=1e-9)


def test_intercept_only_gives_sample_median():
    rng = np.random.default_rng(12)
    for n in [5, 11, 101]:
        y = rng.standard_normal(n) * 4 + 2
        X = np.ones((n, 1))
        o = oracle.default_opts(lambda_min_floor=1e-9)
        r = oracle.fit_path(X, y, [0.0], opts=o)
        assert abs(r["b"][0, 0] - np.median(y)) < 1e-9


# ---------------------------------------------------------------- invariances

def test_invariances():
    rng = np.random.default_rng(21)
    X, y = rand_problem(rng, 80, 5)
    lam = 0.1 * oracle.lambda_max(X, y)
    base = oracle.fit_path(X, y, [lam])
    b0, f0 = base["b"][0], base["f"][0]
    perm = rng.permutation(80)
    r = oracle.fit_path(X[perm], y[perm], [lam])
    assert rel(r["f"][0], f0) < 1e-12
    np.testing.assert_allclose(r["b"][0], b0, atol=1e-9)
    cp = rng.permutation(5)
    r = oracle.fit_path(X[:, cp], y, [lam])
    np.testing.assert_allclose(r["b"][0], b0[cp], atol=1e-9)
    # F is positively homogeneous of degree one in (y, b): scaling y by c
    # with lambda fixed scales the minimiser by c ...
    c = 3.7
    r = oracle.fit_path(X, c * y, [lam])
    np.testing.assert_allclose(r["b"][0], c * b0, atol=1e-8)
    # ... and scaling (X, y, lambda) together leaves it unchanged
    r = oracle.fit_path(c * X, c * y, [c * lam])
    np.testing.assert_allclose(r["b"][0], b0, atol=1e-9)
    # a duplicated row equals that row with weight 2 (row and target doubled)
    Xd = np.vstack([X, X[:1]])
    yd = np.concatenate([y, y[:1]])
    Xw = X.copy()
    yw = y.copy()
    Xw[0] *= 2
    yw[0] *= 2
    fd = oracle.simplex(Xd, yd, lam)[0]
    fw = oracle.simplex(Xw, yw, lam)[0]
    assert rel(fd, fw) < 1e-11
    rd = oracle.fit_path(Xd, yd, [lam])
    assert rel(rd["f"][0], fd) < 1e-11


def test_sign_symmetries_and_a_zero_column():
    rng = np.random.default_rng(23)
    X, y = rand_problem(rng, 70, 5)
    lam = 0.2 * oracle.lambda_max(X, y)
    b0 = oracle.fit_path(X, y, [lam])["b"][0]
    # F(b; X, y) with column j negated equals F with b_j negated
    Xf = X.copy()
    Xf[:, 2] *= -1
    bf = oracle.fit_path(Xf, y, [lam])["b"][0]
    np.testing.assert_allclose(bf, b0 * np.array([1, 1, -1, 1, 1]), atol=1e-9)
    # F(b; X, -y) = F(-b; X, y)
    np.testing.assert_allclose(oracle.fit_path(X, -y, [lam])["b"][0], -b0, atol=1e-9)
    # a column of zeros gets a zero coefficient and changes nothing else
    Xz = np.hstack([X[:, :3], np.zeros((70, 1)), X[:, 3:]])
    bz = oracle.fit_path(Xz, y, [lam])["b"][0]
    assert bz[3] == 0.0
    np.testing.assert_allclose(np.delete(bz, 3), b0, atol=1e-9)


def test_optimum_along_lambda_is_nondecreasing_and_concave():
    # F*(lambda) = min_b (sum |r| + lambda |b|_1) is a minimum of functions
    # affine in lambda: nondecreasing and concave; the minimiser's |b|_1 is
    # its slope, so it does not increase with lambda.  Values from the dense
    # simplex, coefficients from the method's path.
    rng = np.random.default_rng(25)
    X, y = rand_problem(rng, 50, 4)
    lams = oracle.lambda_max(X, y) * np.linspace(0.02, 1.2, 13)
    f = np.array([oracle.simplex(X, y, lam)[0] for lam in lams])
    assert np.all(np.diff(f) >= -1e-9)
    slopes = np.diff(f) / np.diff(lams)
    assert np.all(np.diff(slopes) <= 1e-9)
    path = oracle.fit_path(X, y, lams[::-1])  # descending, warm-started
    l1 = np.abs(path["b"]).sum(axis=1)[::-1]
    assert np.all(np.diff(l1) <= 1e-9)
    np.testing.assert_allclose(path["f"][::-1], f, rtol=1e-10)
    # between grid points the slope of F* brackets |b|_1
    assert np.all(slopes <= l1[:-1] + 1e-9) and np.all(slopes >= l1[1:] - 1e-9)


def test_non_unique_optima_are_flagged():
    # a duplicated column: only b_0 + b_1 matters to the residual and, with
    # equal signs, to the penalty, so every such split of the optimum is
    # optimal (brute force finds several optimal vertices).  The method must
    # flag it NONUNIQUE and the certificate must deny uniqueness, both at the
    # vertex returned and at the midpoint of two optimal vertices (an optimal
    # point that is no vertex: fewer zero residuals than nonzero coefficients)
    rng = np.random.default_rng(31)
    n = 30
    x, z = rng.standard_normal(n), rng.standard_normal(n)
    X = np.column_stack([x, x, z])
    y = 2.0 * x - z + rng.laplace(0, 0.3, n)
    lam = 0.1 * oracle.lambda_max(X, y)
    fb, bb, nd = oracle.brute_force(X, y, lam)
    assert nd > 1
    r = oracle.fit_path(X, y, [lam])
    assert rel(r["f"][0], fb) < 1e-11
    assert r["status"][0] & oracle.FIT_NONUNIQUE
    gap, info = oracle.certify(X, y, r["b"][0], lam)
    assert gap < 1e-9 and not info["unique"]
    s01 = r["b"][0][0] + r["b"][0][1]
    mid = np.array([s01 / 2, s01 / 2, r["b"][0][2]])
    assert rel(F(X, y, mid, lam), fb) < 1e-11  # the optimal set is convex
    gap, info = oracle.certify(X, y, mid, lam)
    assert gap < 1e-9 and not info["unique"]
    # without the duplicate the optimum is a strict vertex and is not flagged
    ru = oracle.fit_path(X[:, [0, 2]], y, [lam])
    assert ru["status"][0] == oracle.FIT_OK
    assert oracle.certify(X[:, [0, 2]], y, ru["b"][0], lam)[1]["unique"]


# ---------------------------------------------------------------- certificate

def test_certificate_detects_suboptimal_points():
    rng = np.random.default_rng(31)
    X, y = rand_problem(rng, 60, 5)
    lam = 0.05 * oracle.lambda_max(X, y)
    fs, bs = oracle.simplex(X, y, lam)
    gap, info = oracle.certify(X, y, bs, lam)
    assert gap < 1e-9
    for trial in range(5):
        bp = bs + rng.standard_normal(5) * 0.05
        gp, _ = oracle.certify(X, y, bp, lam)
        # weak duality: the gap bounds F(b) - F* from above
        assert gp >= F(X, y, bp, lam) - fs - 1e-9
        assert gp > 1e-6


def test_plain_ccd_stalls_but_method_does_not():
    # Section 3.3: coordinate descent alone stops at axis-wise minima.
    rng = np.random.default_rng(41)
    stalls = 0
    for trial in range(6):
        X, y = rand_problem(rng, 100, 8)
        lam = 0.02 * oracle.lambda_max(X, y)
        fs, _ = oracle.simplex(X, y, lam)
        bc, _ = oracle.ccd(X, y, lam)
        if F(X, y, bc, lam) > fs * (1 + 1e-9):
            stalls += 1
        r = oracle.fit_path(X, y, [lam])
        assert rel(r["f"][0], fs) < 1e-11
    assert stalls >= 1


def test_chop_only_variant_is_not_always_optimal_but_never_worse():
    # without the polish the method ends with coordinate descent after the
    # chop (Sections 3.3-3.5): its point is never worse than plain CCD's and
    # is itself an axis-wise minimum of F, so descent from it does not move
    rng = np.random.default_rng(43)
    for trial in range(8):
        X, y = rand_problem(rng, 60, 6)
        lam = 0.05 * oracle.lambda_max(X, y)
        bc, _ = oracle.ccd(X, y, lam)
        o = oracle.default_opts(polish=0)
        r = oracle.fit_path(X, y, [lam], opts=o)
        assert r["f"][0] <= F(X, y, bc, lam) * (1 + 1e-12)
        again, _ = oracle.ccd(X, y, lam, b0=r["b"][0])
        np.testing.assert_allclose(again, r["b"][0], atol=1e-9)


@pytest.mark.parametrize("sections", [3, 4])
def test_chop_is_exact_on_two_coordinates(sections):
    # p = 2: a probe's restricted descent is an exact 1-D minimisation over
    # the other coordinate, so g(t) is the convex partial minimum and both
    # the ternary chop (3 sections) and the four-section "quadrature"
    # reading close in on the global minimum (Sections 3.4-3.5); no polish.
    rng = np.random.default_rng(47)
    ran = 0
    for trial in range(12):
        X = rng.standard_normal((30, 2))
        X[:, 1] = 0.9 * X[:, 0] + 0.3 * X[:, 1]  # correlated axes stall CCD
        y = X @ np.array([1.5, -2.0]) + rng.laplace(0, 0.5, 30)
        lam = 0.05 * oracle.lambda_max(X, y)
        fb, _, _ = oracle.brute_force(X, y, lam)
        o = oracle.default_opts(polish=0, chop_sections=sections, chop_tol=1e-13,
                                chop_max_probes=400, chop_max_extend=80)
        r = oracle.fit_path(X, y, [lam], opts=o)
        ran += r["stats"][0]["chop_ran"]
        assert rel(r["f"][0], fb) < 1e-9, (trial, r["f"][0], fb)
    assert ran >= 2


# ---------------------------------------------------------------- gradient

def test_active_set_gradient_matches_finite_differences():
    rng = np.random.default_rng(51)
    n, nv, p = 60, 20, 4
    Xa = rng.standard_normal((n + nv, p))
    bt = np.array([1.5, 0, -2, 0.0])
    ya = Xa @ bt + rng.laplace(0, 1, n + nv)
    X, y, Xv, yv = Xa[:n], ya[:n], Xa[n:], ya[n:]
    lam = 0.1 * oracle.lambda_max(X, y)

    def loss(X_, y_, lam_):
        r = oracle.fit_path(X_, y_, [lam_])
        return np.abs(yv - Xv @ r["b"][0]).sum(), r

    L0, r0 = loss(X, y, lam)
    g = oracle.grad(X, y, r0["b"][0], r0["basis"][0], Xv, yv)
    assert g["ok"]
    h = 1e-3
    checked = 0
    # y entries
    for i in range(n):
        yp, ym = y.copy(), y.copy()
        yp[i] += h
        ym[i] -= h
        Lp, rp = loss(X, yp, lam)
        Lm, rm = loss(X, ym, lam)
        if sorted(rp["basis"][0]) != sorted(r0["basis"][0]) or \
           sorted(rm["basis"][0]) != sorted(r0["basis"][0]):
            continue  # not a generic point: the vertex changes within h
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g["gy"][i]) <= 1e-3 * max(1, abs(fd)), (i, fd, g["gy"][i])
        checked += 1
    # X entries of basis rows
    for i in set(int(c) for c in r0["basis"][0] if c >= 0):
        for j in range(p):
            Xp, Xm = X.copy(), X.copy()
            Xp[i, j] += h
            Xm[i, j] -= h
            Lp, rp = loss(Xp, y, lam)
            Lm, rm = loss(Xm, y, lam)
            if sorted(rp["basis"][0]) != sorted(r0["basis"][0]) or \
               sorted(rm["basis"][0]) != sorted(r0["basis"][0]):
                continue
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - g["gX"][i, j]) <= 1e-3 * max(1, abs(fd))
            checked += 1
    # lambda: zero at a generic vertex
    Lp, _ = loss(X, y, lam + h)
    Lm, _ = loss(X, y, lam - h)
    assert abs((Lp - Lm) / (2 * h) - g["glam"]) < 1e-6
    # validation rows (direct terms)
    for v in range(3):
        yvp = yv.copy()
        yvp[v] += h
        fd = (np.abs(yvp - Xv @ r0["b"][0]).sum() - L0) / h
        assert abs(fd - g["gyv"][v]) < 1e-6
    # validation design entries (direct terms): central differences, at
    # rows whose residual does not change sign within the step
    bb = r0["b"][0]
    rv = yv - Xv @ bb
    nchk = 0
    for v in range(nv):
        if abs(rv[v]) <= 2 * h * np.abs(bb).sum():
            continue
        for j in range(p):
            Xp, Xm = Xv.copy(), Xv.copy()
            Xp[v, j] += h
            Xm[v, j] -= h
            fd = (np.abs(yv - Xp @ bb).sum() - np.abs(yv - Xm @ bb).sum()) / (2 * h)
            assert abs(fd - g["gXv"][v, j]) < 1e-6, (v, j, fd, g["gXv"][v, j])
            nchk += 1
    assert nchk >= p * nv // 2
    # the upstream derivative scales every output
    g2 = oracle.grad(X, y, bb, r0["basis"][0], Xv, yv, up=-2.5)
    for k in ("gy", "gX", "gyv", "gXv"):
        np.testing.assert_allclose(g2[k], -2.5 * g[k], rtol=1e-12, atol=1e-12)
    assert checked >= n // 2


# ---------------------------------------------------------------- batch API

def test_fit_batch_matches_single_fits():
    batch = synth.batched_like(6, 30, 80, 2, 6, R=120, P=8, seed=5)
    lm = np.array([oracle.lambda_max(*oracle.problem(batch, q)) for q in range(6)])
    lams = lm[:, None] * np.logspace(0, -2, 3)[None, :]
    res = oracle.fit_batch(batch, lams, nthreads=2)
    for q in range(6):
        Xq, yq = oracle.problem(batch, q)
        r = oracle.fit_path(Xq, yq, lams[q])
        np.testing.assert_array_equal(res["b"][q, :, :Xq.shape[1]], r["b"])
        np.testing.assert_array_equal(res["f"][q], r["f"])


def test_bad_lambda_status():
    rng = np.random.default_rng(2)
    X, y = rand_problem(rng, 20, 3)
    r = oracle.fit_path(X, y, [1.0, -1.0, np.nan, 0.5])
    assert list(r["status"][[1, 2]]) == [oracle.FIT_BAD_INPUT] * 2
    assert np.all(r["b"][1:3] == 0)
    assert r["status"][3] in (0, oracle.FIT_NONUNIQUE)


def test_exact_finish_makes_the_result_independent_of_chop_settings():
    # the vertex polish certifies the LP optimum whatever the chop did (or
    # whether it ran), so the optimum value does not depend on the chop's
    # hyper-parameters or the descent tolerance; each setting also matches
    # the dense simplex
    rng = np.random.default_rng(21)
    settings = [dict(), dict(chop=0), dict(chop_sections=4), dict(tol_move=1e-3),
                dict(chop=0, tol_move=1e-3), dict(chop_max_probes=2, probe_max_sweeps=1),
                # the chop constants proposed as readings of Sections 3.4-3.5
                # before the exact finish existed: a bracket of max(1, |b_k|),
                # up to 40 extensions, range 1e-12 or 80 probes
                dict(chop_bracket=1.0, chop_max_extend=40, chop_tol=1e-12, chop_max_probes=80)]
    for n, p in [(40, 3), (120, 6), (300, 10)]:
        X, y = rand_problem(rng, n, p)
        lams = oracle.lambda_max(X, y) * np.array([0.5, 0.1, 0.01])
        ref = [oracle.simplex(X, y, lam)[0] for lam in lams]
        for kw in settings:
            r = oracle.fit_path(X, y, lams, opts=oracle.default_opts(**kw))
            assert np.all((r["status"] & oracle.FIT_MAX_ITERS) == 0), kw
            for l in range(len(lams)):
                assert rel(r["f"][l], ref[l]) < 1e-10, (n, p, kw, l)

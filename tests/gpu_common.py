"""Helpers shared by the GPU tests: run the CUDA path and compare with the
FP64 oracle.  Parity bar (per fit, problem q at path position l):
  rel. objective error |F(b_gpu) - F*| / F* <= 1e-5   (F evaluated in FP64)
  same support {j : b_j != 0} when the oracle's optimum is unique at
      float32 resolution
  max_j |b_gpu - b*| <= 1e-4 * max(1, |b*|_inf)      there too
where F* and b* come from the oracle on the same float32 inputs and the
same float32 lambdas, converted to float64.

"Unique at float32 resolution": the oracle's certificate shows a strict
vertex, its support is the same at lambda * (1 -+ LAM_REL), and every
multiplier of its basis keeps a slack to its cap (1 for a row, lambda for a
coordinate) larger than the kernel could misjudge (margin_needed):

  the kernel's multipliers solve B^T mu = -g with the column sums
  g_c = -sum_{rows off the basis} sign(r_i) x_ic formed in float32
  (per-thread compensated sums, a 5-level butterfly, changed rows added
  in batches).  The first-order error of such sums is at most
  K_SUM * u * sum_i |x_ic| (u = 2^-24: 2u for a compensated sum, 5u for
  the butterfly, the rest for the batched updates); through the solve it
  becomes |B^-T| (K_SUM * u * sum_i |x_i|) per multiplier, and the kernel
  accepts a multiplier up to tol_opt * max(1, lambda) beyond its cap.
  A slack above (that error + that tolerance) / cap for every multiplier
  means the kernel must judge the oracle's vertex as the oracle does.

Otherwise the optimum is degenerate to within float32 resolution (several
vertices reach F* to within 1e-5, or a breakpoint of the solution path lies
within float32 rounding of lambda), so only the objective -- the one unique
quantity -- is compared there.  compare() counts both kinds of fit."""
import numpy as np

import oracle

REL_OBJ = 1e-5
REL_COEF = 1e-4
LAM_REL = 2e-6  # float32 multiplier sums over 1e4 rows carry ~1e-6 relative error
U32 = 2.0 ** -24
K_SUM = 16
TOL_OPT_GPU = 2e-5  # the library's default tol_opt


def basis_matrix(X, codes):
    """Rows of the basis: x_i for a row code i >= 0, e_j for code -(j+1)."""
    p = X.shape[1]
    B = np.zeros((p, p))
    for k, cd in enumerate(codes):
        if cd >= 0:
            B[k] = X[cd]
        else:
            B[k, -cd - 1] = 1.0
    return B


def margin_needed(X, lam, codes, tol_opt=TOL_OPT_GPU):
    """Smallest normalised multiplier slack the kernel's float32 arithmetic
    cannot misjudge at the basis `codes` (module docstring); inf for a
    singular basis."""
    B = basis_matrix(X, codes)
    try:
        binv_t = np.linalg.inv(B.T)
    except np.linalg.LinAlgError:
        return np.inf
    dg = K_SUM * U32 * np.abs(X).sum(axis=0)
    dmu = np.abs(binv_t) @ dg
    cap = np.where(np.asarray(codes) >= 0, 1.0, lam)
    return float(np.max((dmu + tol_opt * max(1.0, lam)) / np.maximum(cap, 1e-300)))


def exact_problems(seed, count=40):
    """Problems on which float32 arithmetic is exact for the descent and
    the four-section chop: X in {-1, 0, 1}, integer targets in [-15, 15],
    integer lambda, so every key b_j + r_i / x_ij, residual and weight sum
    is an integer or a dyadic rational of few bits; with a dyadic chop
    bracket (1/16) and tolerance (2^-10) every probe point is dyadic too,
    and the objectives (a few hundred, few fractional bits) are exact.
    Returns ([(X [n, p] float32, y [n] float32)], lambdas [count, 1])."""
    rng = np.random.default_rng(seed)
    probs, lams = [], []
    for t in range(count):
        n = int(rng.integers(30, 160))
        p = int(rng.integers(3, 9))
        X = rng.choice(np.array([-1.0, 0.0, 1.0]), size=(n, p), p=[0.4, 0.2, 0.4])
        bt = np.zeros(p)
        bt[rng.choice(p, 2, replace=False)] = rng.integers(-4, 5, 2)
        y = np.clip(X @ bt + np.round(rng.laplace(0, 2, n)), -15, 15)
        probs.append((X.astype(np.float32), y.astype(np.float32)))
        lams.append(float(max(1, round(0.1 * oracle.lambda_max(X, y)))))
    return probs, np.array(lams, np.float32)[:, None]


def well_separated(X, y, b, codes, lam, opts=None):
    """The oracle's optimum b (basis `codes`) is unique at float32
    resolution (module docstring): a strict vertex whose multipliers keep
    more slack than margin_needed, with the same support at
    lambda * (1 -+ LAM_REL)."""
    _, info = oracle.certify(X, y, b, lam)
    margin = min(1.0 - info["u_e_max"], 1.0 - info["c_off_max"])
    if not info["unique"] or margin < margin_needed(X, lam, codes):
        return False
    sup = b != 0
    return all(np.array_equal(oracle.fit_path(X, y, [lam * (1.0 + sg * LAM_REL)],
                                              b_init=b, opts=opts)["b"][0] != 0, sup)
               for sg in (-1.0, 1.0))


EXACT_CHOP_OPTS = dict(polish=0, chop_sections=4, chop_bracket=0.0625, chop_tol=2.0 ** -10)


def compare(batch, lam, b_gpu, obj_gpu, status_gpu, problems=None, opts=None):
    """Returns a dict of counts and the worst errors; asserts nothing.
    `support_checked` fits were compared on support and coefficients,
    `objective_only` fits (degenerate at float32 resolution) on the
    objective alone."""
    lam = np.asarray(lam, np.float64)
    qs = range(lam.shape[0]) if problems is None else problems
    worst_obj = 0.0
    worst_coef = 0.0
    bad = []
    checked = support_checked = objective_only = 0
    for q in qs:
        X, y = oracle.problem(batch, q)
        p = X.shape[1]
        ref = oracle.fit_path(X, y, lam[q], opts=opts)
        for l in range(lam.shape[1]):
            checked += 1
            if ref["status"][l] & oracle.FIT_BAD_INPUT:
                if not (status_gpu[q, l] & 2):
                    bad.append((q, l, "status"))
                continue
            bg = np.asarray(b_gpu[q, l, :p], np.float64)
            fo = ref["f"][l]
            fg = oracle.objective(X, y, bg, lam[q, l])
            eo = abs(fg - fo) / max(1.0, fo)
            worst_obj = max(worst_obj, eo)
            if eo > REL_OBJ:
                bad.append((q, l, "obj", eo))
            if abs(obj_gpu[q, l] - fg) > 1e-5 * max(1.0, fg):
                bad.append((q, l, "obj_out", obj_gpu[q, l], fg))
            unique = not (ref["status"][l] & oracle.FIT_NONUNIQUE) and \
                well_separated(X, y, ref["b"][l], ref["basis"][l], lam[q, l], opts)
            if unique:
                support_checked += 1
                if not np.array_equal(bg != 0, ref["b"][l] != 0):
                    bad.append((q, l, "support"))
                ec = np.max(np.abs(bg - ref["b"][l])) / max(1.0, np.max(np.abs(ref["b"][l])))
                worst_coef = max(worst_coef, ec)
                if ec > REL_COEF:
                    bad.append((q, l, "coef", ec))
            else:
                objective_only += 1
            if np.any(b_gpu[q, l, p:] != 0):
                bad.append((q, l, "padding"))
    return dict(bad=bad, worst_obj=worst_obj, worst_coef=worst_coef, checked=checked,
                support_checked=support_checked, objective_only=objective_only)


def _compare_chunk(args):
    batch, lam, b_gpu, obj_gpu, status_gpu, problems, opts = args
    return compare(batch, lam, b_gpu, obj_gpu, status_gpu, problems=problems, opts=opts)


def compare_parallel(batch, lam, b_gpu, obj_gpu, status_gpu, problems, opts=None, workers=8):
    """compare() over `problems` split across worker processes (started by
    spawn, so safe after CUDA has been initialised in this process); merges
    the counts and worst errors."""
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    problems = list(problems)
    w = max(1, min(workers, os.cpu_count() or 1, len(problems)))
    chunks = [problems[k::w] for k in range(w)]
    jobs = [(batch, lam, b_gpu, obj_gpu, status_gpu, c, opts) for c in chunks if c]
    with ProcessPoolExecutor(max_workers=len(jobs), mp_context=mp.get_context("spawn")) as ex:
        parts = list(ex.map(_compare_chunk, jobs))
    return dict(bad=[x for r in parts for x in r["bad"]],
                worst_obj=max(r["worst_obj"] for r in parts),
                worst_coef=max(r["worst_coef"] for r in parts),
                checked=sum(r["checked"] for r in parts),
                support_checked=sum(r["support_checked"] for r in parts),
                objective_only=sum(r["objective_only"] for r in parts))

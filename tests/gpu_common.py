"""Helpers shared by the GPU tests: run the CUDA path and compare with the
FP64 oracle.  Parity bar (per fit, problem q at path position l):
  rel. objective error |F(b_gpu) - F*| / F* <= 1e-5   (F evaluated in FP64)
  same support {j : b_j != 0} when the oracle's optimum is unique
  max_j |b_gpu - b*| <= 1e-4 * max(1, |b*|_inf)      when unique
where F* and b* come from the oracle on the same float32 inputs and the
same float32 lambdas, converted to float64.

"Unique" means the oracle's certificate shows a strict vertex whose
complementarity margin (1 - max|u_E|, 1 - max_off |X^T u|/lambda) is at
least MARGIN, and whose support is the same at lambda * (1 -+ LAM_REL).
Otherwise the optimum is degenerate to within float32 resolution: several
vertices reach F* to within 1e-5, or a breakpoint of the solution path
lies within float32 rounding of lambda (e.g. lambda rounded a few ulp
below lambda_max, where the FP64 optimum carries a coefficient of order
(lambda_max - lambda) / lambda), so only the objective -- the one unique
quantity -- is compared there."""
import numpy as np

import oracle

REL_OBJ = 1e-5
REL_COEF = 1e-4
MARGIN = 1e-4
LAM_REL = 2e-6  # float32 multiplier sums over 1e4 rows carry ~1e-6 relative error


def compare(batch, lam, b_gpu, obj_gpu, status_gpu, problems=None, opts=None):
    """Returns a dict of counts and the worst errors; asserts nothing."""
    lam = np.asarray(lam, np.float64)
    qs = range(lam.shape[0]) if problems is None else problems
    worst_obj = 0.0
    worst_coef = 0.0
    bad = []
    checked = 0
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
            unique = not (ref["status"][l] & oracle.FIT_NONUNIQUE)
            if unique:
                _, info = oracle.certify(X, y, ref["b"][l], lam[q, l])
                margin = min(1.0 - info["u_e_max"], 1.0 - info["c_off_max"])
                unique = info["unique"] and margin >= MARGIN
            if unique:
                sup = ref["b"][l] != 0
                for sg in (-1.0, 1.0):
                    alt = oracle.fit_path(X, y, [lam[q, l] * (1.0 + sg * LAM_REL)],
                                          b_init=ref["b"][l], opts=opts)
                    unique = unique and np.array_equal(alt["b"][0] != 0, sup)
            if unique:
                if not np.array_equal(bg != 0, ref["b"][l] != 0):
                    bad.append((q, l, "support"))
                ec = np.max(np.abs(bg - ref["b"][l])) / max(1.0, np.max(np.abs(ref["b"][l])))
                worst_coef = max(worst_coef, ec)
                if ec > REL_COEF:
                    bad.append((q, l, "coef", ec))
            if np.any(b_gpu[q, l, p:] != 0):
                bad.append((q, l, "padding"))
    return dict(bad=bad, worst_obj=worst_obj, worst_coef=worst_coef, checked=checked)


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
                checked=sum(r["checked"] for r in parts))

"""FP64 CPU oracle for batched LAD-LASSO (test infrastructure only).

Only tests/, the package smoke check and the CPU-baseline leg of bench.py
may import this module.  The product path (the CUDA library and its
binding) never imports, links or runs anything here; the two share no code.

This is a thin ctypes wrapper over `ladlasso_oracle.c` (plain C, double
precision).  Each function names the part of the paper it restates; the C
source carries the details.  Inputs are numpy arrays; a problem's design is
gathered here, in numpy, from the shared-X batch layout of
`paper_2510_15649_gb300.synth`.

Parity status of each function (what pins it in tests/test_oracle.py):
  axis update     brute force over 1-D breakpoints; closed form for p = 1
  ccd/chop/polish F equal to brute force (Section 3.2) and to the dense
                  simplex (Section 3.1) on tiny problems; certificate gap
  brute_force     equal to simplex; closed-form special cases
  simplex         equal to brute force; scipy's HiGHS LP as an outside check
  certify         zero gap at LP optima, positive gap at perturbed points
  lambda_max      b = 0 optimal at lambda_max, not below (simplex)
  grad            central finite differences of refits at generic points
                  (training y and X rows), of the loss itself (validation
                  y and X rows); exact scaling by the upstream factor
Each of 51 planted mistakes in the C source fails at least one of these
pins (tests/test_oracle_mutants.py).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ladlasso_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lib = None

FIT_OK, FIT_MAX_ITERS, FIT_BAD_INPUT, FIT_NONUNIQUE = 0, 1, 2, 4


class Opts(C.Structure):
    _fields_ = [("tol_move", C.c_double), ("max_sweeps", C.c_int),
                ("chop", C.c_int), ("chop_bracket", C.c_double),
                ("chop_tol", C.c_double), ("chop_max_probes", C.c_int),
                ("chop_max_extend", C.c_int), ("probe_max_sweeps", C.c_int),
                ("polish", C.c_int), ("max_pivots", C.c_int),
                ("tol_opt", C.c_double), ("lambda_min_floor", C.c_double),
                ("chop_sections", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("sweeps", C.c_int), ("probes", C.c_int), ("extends", C.c_int),
                ("pivots", C.c_int), ("ccd_optimal", C.c_int),
                ("chop_ran", C.c_int), ("chop_optimal", C.c_int)]


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(C.CDLL(_LIB))
    return _lib


def use_library(path: str) -> None:
    """Run every oracle function from the shared library at `path`, built
    from a modified copy of ladlasso_oracle.c (the tests that plant a
    mistake in the oracle to show that its pins catch it)."""
    global _lib
    _lib = _bind(C.CDLL(path))


def _bind(lib):
    """Declare the argument and result types of the C entry points."""
    D, I, P = C.c_double, C.c_int, C.c_void_p
    lib.orc_default_opts.argtypes = [C.POINTER(Opts)]
    lib.orc_objective.restype = D
    lib.orc_objective.argtypes = [I, I, P, P, P, D]
    lib.orc_axis_update.restype = D
    lib.orc_axis_update.argtypes = [I, I, P, P, P, D, I, C.POINTER(I), P]
    lib.orc_ccd.restype = I
    lib.orc_ccd.argtypes = [I, I, P, P, P, D, I, D, I, P, P]
    lib.orc_fit_path.restype = None
    lib.orc_fit_path.argtypes = [I, I, P, P, I, P, P, C.POINTER(Opts), P, P, P, P, P]
    lib.orc_fit_batch.restype = I
    lib.orc_fit_batch.argtypes = [I, P, P, P, P, P, P, I, I, P, C.POINTER(Opts), P, P, P, I]
    lib.orc_lambda_max.restype = D
    lib.orc_lambda_max.argtypes = [I, I, P, P]
    lib.orc_brute_force.restype = D
    lib.orc_brute_force.argtypes = [I, I, P, P, D, P, C.POINTER(I)]
    lib.orc_simplex.restype = D
    lib.orc_simplex.argtypes = [I, I, P, P, D, P, I]
    lib.orc_certify.restype = D
    lib.orc_certify.argtypes = [I, I, P, P, P, D, D, D, P]
    lib.orc_grad.restype = I
    lib.orc_grad.argtypes = [I, I, P, P, P, P, I, P, P, D, P, P, P, P, P]
    return lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def default_opts(**kw) -> Opts:
    """Default method options (the paper's speed/accuracy hyper-parameters,
    Section 5, plus the polish controls); keyword overrides allowed."""
    o = Opts()
    _load().orc_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def objective(X, y, b, lam) -> float:
    X, y, b = _d(X), _d(y), _d(b)
    n, p = X.shape
    return _load().orc_objective(n, p, _ptr(X), _ptr(y), _ptr(b), float(lam))


def axis_update(X, y, b, lam, j):
    """One exact axis minimisation (Section 3.3).  Returns (b_new, r_new, piv)."""
    X, b = _d(X), _d(b).copy()
    n, p = X.shape
    r = _d(y) - X @ b
    work = np.empty(3 * (n + p + 1), np.float64)  # >= sizeof(bp_t)*(n+1)
    piv = C.c_int(0)
    _load().orc_axis_update(n, p, _ptr(X), _ptr(b), _ptr(r), float(lam), int(j),
                            C.byref(piv), _ptr(work))
    return b, r, piv.value


def ccd(X, y, lam, b0=None, tol_move=1e-12, max_sweeps=1000, skip=-1):
    """Cyclical coordinate descent to an axis-wise fixed point (Section 3.3).
    Returns (b, sweeps) -- sweeps negative when the cap was hit."""
    X = _d(X)
    n, p = X.shape
    b = np.zeros(p) if b0 is None else _d(b0).copy()
    r = _d(y) - X @ b
    piv = np.zeros(p, np.int32)
    work = np.empty(3 * (n + p + 1), np.float64)
    s = _load().orc_ccd(n, p, _ptr(X), _ptr(b), _ptr(r), float(lam), int(skip),
                        float(tol_move), int(max_sweeps), _ptr(piv), _ptr(work))
    return b, s


def fit_path(X, y, lambdas, b_init=None, opts: Opts | None = None):
    """Full method on one problem along a lambda path (warm starts).
    Returns dict(b [L,p], f [L], status [L], basis [L,p], stats list)."""
    X, y = _d(X), _d(y)
    n, p = X.shape
    lam = _d(np.atleast_1d(lambdas))
    L = lam.size
    o = opts or default_opts()
    b_out = np.zeros((L, p))
    f_out = np.zeros(L)
    st_out = np.zeros(L, np.int32)
    basis = np.zeros((L, p), np.int32)
    stats = (Stats * L)()
    bi = None if b_init is None else _d(b_init)
    _load().orc_fit_path(n, p, _ptr(X), _ptr(y), L, _ptr(lam),
                         None if bi is None else _ptr(bi), C.byref(o),
                         _ptr(b_out), _ptr(f_out), _ptr(st_out), _ptr(basis),
                         C.cast(stats, C.c_void_p))
    return dict(b=b_out, f=f_out, status=st_out, basis=basis,
                stats=[{k: getattr(s, k) for k, _ in Stats._fields_} for s in stats])


def problem(batch: dict, q: int):
    """Problem q of a batch as (X_q [n,p] float64, y_q [n] float64)."""
    o0, o1 = int(batch["offsets"][q]), int(batch["offsets"][q + 1])
    p = int(batch["p"][q])
    rows = np.arange(o0, o1) if batch.get("row_idx") is None else batch["row_idx"][o0:o1]
    return (np.asarray(batch["X"], np.float64)[rows, :p],
            np.asarray(batch["y"], np.float64)[o0:o1])


def fit_batch(batch: dict, lambdas, problems=None, opts: Opts | None = None,
              nthreads: int = 0):
    """Fit many problems (OpenMP over problems).  lambdas: [B, L].
    Returns dict(b [B,L,P], f [B,L], status [B,L], threads)."""
    qs = np.arange(len(batch["p"])) if problems is None else np.asarray(problems)
    lam = np.asarray(lambdas, np.float64)[qs]
    B, L = lam.shape
    P = int(np.max(batch["p"][qs])) if B else 0
    Xs, ys, ns, ps = [], [], [], []
    for q in qs:
        Xq, yq = problem(batch, int(q))
        Xs.append(Xq.ravel())
        ys.append(yq)
        ns.append(Xq.shape[0])
        ps.append(Xq.shape[1])
    xoff = np.zeros(B, np.int64)
    yoff = np.zeros(B, np.int64)
    if B:
        xoff[1:] = np.cumsum([x.size for x in Xs])[:-1]
        yoff[1:] = np.cumsum(ns)[:-1]
    Xc = _d(np.concatenate(Xs)) if B else np.zeros(1)
    yc = _d(np.concatenate(ys)) if B else np.zeros(1)
    n_a = np.asarray(ns, np.int32)
    p_a = np.asarray(ps, np.int32)
    lam = _d(lam)
    b_out = np.zeros((B, L, P))
    f_out = np.zeros((B, L))
    st = np.zeros((B, L), np.int32)
    o = opts or default_opts()
    used = _load().orc_fit_batch(B, _ptr(Xc), _ptr(xoff), _ptr(yc), _ptr(yoff),
                                 _ptr(n_a), _ptr(p_a), P, L, _ptr(lam), C.byref(o),
                                 _ptr(b_out), _ptr(f_out), _ptr(st), int(nthreads))
    return dict(b=b_out, f=f_out, status=st, threads=used)


def lambda_max(X, y) -> float:
    """Smallest lambda at which b = 0 is optimal: |X^T sign(y)|_inf."""
    X, y = _d(X), _d(y)
    n, p = X.shape
    return _load().orc_lambda_max(n, p, _ptr(X), _ptr(y))


def brute_force(X, y, lam):
    """Section 3.2: min of F over all vertices.  Returns (F*, b, n_distinct)."""
    X, y = _d(X), _d(y)
    n, p = X.shape
    b = np.zeros(p)
    nd = C.c_int(0)
    f = _load().orc_brute_force(n, p, _ptr(X), _ptr(y), float(lam), _ptr(b), C.byref(nd))
    return f, b, nd.value


def simplex(X, y, lam, max_iter=200000):
    """Section 3.1: dense Bland simplex of the split-variable LP.
    Returns (F*, b)."""
    X, y = _d(X), _d(y)
    n, p = X.shape
    b = np.zeros(p)
    f = _load().orc_simplex(n, p, _ptr(X), _ptr(y), float(lam), _ptr(b), int(max_iter))
    return f, b


def certify(X, y, b, lam, eps_r=1e-9, eps_b=1e-12):
    """Duality-gap certificate at b.  Returns (gap, info dict)."""
    X, y, b = _d(X), _d(y), _d(b)
    n, p = X.shape
    out = np.zeros(6)
    gap = _load().orc_certify(n, p, _ptr(X), _ptr(y), _ptr(b), float(lam),
                              float(eps_r), float(eps_b), _ptr(out))
    return gap, dict(dual=out[0], u_e_max=out[1], c_off_max=out[2],
                     n_e=int(out[3]), n_s=int(out[4]), unique=bool(out[5]))


def grad(X, y, b, basis, Xv, yv, up=1.0):
    """Gradient of the validation LAD loss at the final vertex.
    Returns dict(gy, gX, gyv, gXv, glam, ok)."""
    X, y, b, Xv, yv = _d(X), _d(y), _d(b), _d(Xv), _d(yv)
    n, p = X.shape
    nv = Xv.shape[0]
    basis = np.ascontiguousarray(basis, np.int32)
    gy, gX = np.zeros(n), np.zeros((n, p))
    gyv, gXv = np.zeros(nv), np.zeros((nv, p))
    gl = np.zeros(1)
    rc = _load().orc_grad(n, p, _ptr(X), _ptr(y), _ptr(b), _ptr(basis), nv, _ptr(Xv),
                          _ptr(yv), float(up), _ptr(gy), _ptr(gX), _ptr(gyv), _ptr(gXv),
                          _ptr(gl))
    return dict(gy=gy, gX=gX, gyv=gyv, gXv=gXv, glam=float(gl[0]), ok=rc == 0)

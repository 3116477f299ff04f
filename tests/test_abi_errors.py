"""Host-checkable argument errors of the C ABI (include/ladlasso.h): every
call below breaks one documented condition and must return its negative
status before any CUDA work, and empty problem sets (B = 0) return OK.
Buffers are host memory and no call reaches a launch; the module runs only
where no CUDA device exists, so a check that fell through would fail with a
CUDA error instead of touching a GPU."""
import ctypes as C
import math

import numpy as np
import pytest
import torch

from paper_2510_15649_gb300 import build
from paper_2510_15649_gb300 import ladlasso as ll

pytestmark = pytest.mark.skipif(torch.cuda.is_available(),
                                reason="argument checks are exercised only without a device")

INVALID, NOMEM, WORKSPACE = ll.ERR_INVALID, ll.ERR_NOMEM, ll.ERR_WORKSPACE
KMAXP = 256  # largest P_cols the library accepts


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ll.lib()


class Host:
    """A valid problem set of B problems x n rows x P columns in host
    buffers (pointers only; nothing reads them on the host)."""

    def __init__(self, lib, B=1, n=10, P=4, L=2):
        self.B, self.n, self.P, self.L = B, n, P, L
        rows = B * n
        self.X = np.zeros((max(rows, 1), P), np.float32)
        self.y = np.zeros(max(rows, 1), np.float32)
        self.off = np.arange(B + 1, dtype=np.int64) * n
        self.lam = np.zeros(max(B * L, 1), np.float32)
        self.b = np.zeros(max(B * L * P, 1), np.float32)
        self.obj = np.zeros(max(B * L, 1), np.float32)
        self.ws_bytes = lib.ladlasso_workspace_size(B, P, rows, L)
        assert self.ws_bytes > 0
        self.ws_buf = np.zeros(self.ws_bytes + 512, np.uint8)
        base = self.ws_buf.ctypes.data
        self.ws = (base + 255) // 256 * 256
        self.opts = ll.default_opts()
        d = ll.Dims()
        d.B, d.P_cols, d.L, d.n_max = B, P, L, n
        d.ldX, d.rows_X, d.total_rows = P, rows, rows
        d.workspace, d.workspace_bytes = self.ws, self.ws_bytes
        d.opts = C.addressof(self.opts)
        self.d = d

    def args(self, **kw):
        """(X, y, row_idx, offsets, lambdas, b_out, obj_out) pointers, with
        any of them replaced by `kw` (None = NULL)."""
        a = dict(X=self.X.ctypes.data, y=self.y.ctypes.data, row_idx=None,
                 offsets=self.off.ctypes.data, lambdas=self.lam.ctypes.data,
                 b_out=self.b.ctypes.data, obj_out=self.obj.ctypes.data)
        a.update(kw)
        return [a[k] for k in ("X", "y", "row_idx", "offsets", "lambdas", "b_out", "obj_out")]


# one broken condition per case: (dims field overrides, pointer overrides, opts overrides)
SHARED_CASES = {
    "B < 0": ({"B": -1}, {}, {}),
    "L < 1": ({"L": 0}, {}, {}),
    "P_cols < 1": ({"P_cols": 0}, {}, {}),
    "P_cols too large": ({"P_cols": KMAXP + 1, "ldX": KMAXP + 1}, {}, {}),
    "ldX < P_cols": ({"ldX": 3}, {}, {}),
    "rows_X < 0": ({"rows_X": -1}, {}, {}),
    "total_rows < 0": ({"total_rows": -1}, {}, {}),
    "n_max < 0": ({"n_max": -1}, {}, {}),
    "offsets NULL": ({}, {"offsets": None}, {}),
    "y NULL": ({}, {"y": None}, {}),
    "X NULL": ({}, {"X": None}, {}),
    "slots beyond X without row_idx": ({"rows_X": 5}, {}, {}),
    "workspace NULL": ({"workspace": None}, {}, {}),
    "workspace too small": ({"workspace_bytes": -1}, {}, {}),
    "workspace misaligned": ({"workspace": 16}, {}, {}),
    "chop_sections": ({}, {}, {"chop_sections": 2}),
    "max_sweeps": ({}, {}, {"max_sweeps": 0}),
    "tol_move < 0": ({}, {}, {"tol_move": -1.0}),
    "tol_move NaN": ({}, {}, {"tol_move": math.nan}),
    "chop_bracket": ({}, {}, {"chop_bracket": 0.0}),
    "probe_max_sweeps": ({}, {}, {"probe_max_sweeps": 0}),
    "max_pivots < 0": ({}, {}, {"max_pivots": -1}),
    "tol_opt < 0": ({}, {}, {"tol_opt": -1.0}),
    "lambda_min_floor < 0": ({}, {}, {"lambda_min_floor": -1.0}),
}
SHARED_EXPECT = {k: (WORKSPACE if k.startswith("workspace") else INVALID) for k in SHARED_CASES}

FIT_CASES = {
    "lambdas NULL": ({}, {"lambdas": None}, {}),
    "b_out NULL": ({}, {"b_out": None}, {}),
    "obj_out NULL": ({}, {"obj_out": None}, {}),
    "group_threads": ({"group_threads": 96}, {}, {}),
    "fits_per_block < 0": ({"fits_per_block": -1}, {}, {}),
    "work_order 2": ({"work_order": 2}, {}, {}),
    "work_order < 0": ({"work_order": -1}, {}, {}),
}


def _apply(h, dims_kw, opts_kw):
    for k, v in opts_kw.items():
        setattr(h.opts, k, v)
    for k, v in dims_kw.items():
        if k == "workspace":
            v = None if v is None else h.ws + v
        elif k == "workspace_bytes":
            v = h.ws_bytes + v
        setattr(h.d, k, v)


@pytest.mark.parametrize("entry", ["ladlasso_fit_batched", "ladlasso_fit_batched_thread"])
@pytest.mark.parametrize("case", sorted(list(SHARED_CASES) + list(FIT_CASES)))
def test_fit_entry_points_reject_bad_arguments(lib, entry, case):
    h = Host(lib)
    dims_kw, ptr_kw, opts_kw = {**SHARED_CASES, **FIT_CASES}[case]
    _apply(h, dims_kw, opts_kw)
    rc = getattr(lib, entry)(*h.args(**ptr_kw), C.byref(h.d), None)
    assert rc == SHARED_EXPECT.get(case, INVALID), (entry, case, rc)


def test_fit_rejects_rows_beyond_the_one_warp_limit(lib):
    h = Host(lib)
    h.d.group_threads = 32
    h.d.n_max = 1 << 20
    assert lib.ladlasso_fit_batched(*h.args(), C.byref(h.d), None) == NOMEM


@pytest.mark.parametrize("case", sorted(SHARED_CASES))
def test_lambda_max_rejects_bad_arguments(lib, case):
    h = Host(lib)
    dims_kw, ptr_kw, opts_kw = SHARED_CASES[case]
    _apply(h, dims_kw, opts_kw)
    X, y, ri, off, *_ = h.args(**ptr_kw)
    out = np.zeros(1, np.float32)
    assert lib.ladlasso_lambda_max(X, y, ri, off, C.byref(h.d), out.ctypes.data, None) == \
        SHARED_EXPECT[case]


def test_lambda_max_needs_an_output(lib):
    h = Host(lib)
    X, y, ri, off, *_ = h.args()
    assert lib.ladlasso_lambda_max(X, y, ri, off, C.byref(h.d), None, None) == INVALID


def test_lambda_path_rejects_bad_arguments(lib):
    lm = np.ones(4, np.float32)
    out = np.zeros(16, np.float32)
    f = lib.ladlasso_lambda_path
    for B, L, ratio in [(-1, 4, 0.5), (4, 0, 0.5), (4, 4, 0.0), (4, 4, 1.5), (4, 4, math.nan),
                        (4, 4, -0.1)]:
        assert f(lm.ctypes.data, B, L, ratio, out.ctypes.data, None) == INVALID, (B, L, ratio)
    assert f(None, 4, 4, 0.5, out.ctypes.data, None) == INVALID
    assert f(lm.ctypes.data, 4, 4, 0.5, None, None) == INVALID


def test_workspace_size_is_zero_for_invalid_sizes(lib):
    f = lib.ladlasso_workspace_size
    assert f(1, 4, 10, 0) == 0
    assert f(-1, 4, 10, 1) == 0
    assert f(1, 0, 10, 1) == 0
    assert f(1, KMAXP + 1, 10, 1) == 0
    assert f(1, 4, -1, 1) == 0
    # monotone in every size
    assert f(2, 4, 10, 1) > f(1, 4, 10, 1)
    assert f(1, 8, 10, 1) > f(1, 4, 10, 1)
    assert f(1, 4, 1000, 1) > f(1, 4, 10, 1)


@pytest.mark.parametrize("case", ["d NULL", "offsets NULL", "b_out NULL", "loss NULL", "B < 0",
                                  "L < 1", "P_cols too large", "ldX < P_cols", "y NULL",
                                  "slots beyond X without row_idx"])
def test_path_loss_rejects_bad_arguments(lib, case):
    h = Host(lib)
    loss = np.zeros(2, np.float32)
    X, y, ri, off = h.X.ctypes.data, h.y.ctypes.data, None, h.off.ctypes.data
    b, lo, d = h.b.ctypes.data, loss.ctypes.data, C.byref(h.d)
    if case == "d NULL":
        d = None
    elif case == "offsets NULL":
        off = None
    elif case == "b_out NULL":
        b = None
    elif case == "loss NULL":
        lo = None
    elif case == "y NULL":
        y = None
    else:
        dims_kw = {"B < 0": {"B": -1}, "L < 1": {"L": 0},
                   "P_cols too large": {"P_cols": KMAXP + 1, "ldX": KMAXP + 1},
                   "ldX < P_cols": {"ldX": 3},
                   "slots beyond X without row_idx": {"rows_X": 5}}[case]
        _apply(h, dims_kw, {})
    assert lib.ladlasso_path_loss(X, y, ri, off, d, b, lo, None) == INVALID


def _backward(lib, h, **kw):
    nv = 4
    Xv = np.zeros((nv, h.P), np.float32)
    yv = np.zeros(nv, np.float32)
    voff = np.array([0, nv], np.int64)
    basis = np.zeros(h.B * h.L * h.P, np.int32)
    g1 = np.zeros(max(h.B, 1), np.float32)
    gy = np.zeros_like(h.y)
    gX = np.zeros_like(h.X)
    gyv = np.zeros_like(yv)
    gXv = np.zeros_like(Xv)
    a = dict(pos=0, b=h.b.ctypes.data, basis=basis.ctypes.data, Xv=Xv.ctypes.data, ldXv=h.P,
             yv=yv.ctypes.data, voff=voff.ctypes.data, nv=nv, gup=g1.ctypes.data,
             glam=g1.ctypes.data, gy=gy.ctypes.data, gX=gX.ctypes.data, gyv=gyv.ctypes.data,
             gXv=gXv.ctypes.data)
    a.update(kw)
    return lib.ladlasso_fit_backward(
        h.X.ctypes.data, h.y.ctypes.data, None, h.off.ctypes.data, C.byref(h.d), a["pos"],
        a["b"], a["basis"], a["Xv"], a["ldXv"], a["yv"], None, a["voff"], a["nv"], a["gup"],
        a["glam"], a["gy"], a["gX"], a["gyv"], a["gXv"], None, None, None)


@pytest.mark.parametrize("kw", [{"pos": -1}, {"pos": 2}, {"b": None}, {"basis": None},
                                {"voff": None}, {"gup": None}, {"glam": None}, {"gy": None},
                                {"gX": None}, {"gyv": None}, {"gXv": None}, {"nv": -1},
                                {"ldXv": 3}, {"yv": None}, {"Xv": None}],
                         ids=lambda kw: ",".join(f"{k}={v}" for k, v in kw.items()))
def test_backward_rejects_bad_arguments(lib, kw):
    h = Host(lib)
    assert _backward(lib, h, **kw) == INVALID


def test_noalloc_rejects_bad_arguments(lib):
    f = lib.ladlasso_fit_batched_noalloc
    for case in ("offsets NULL", "B < 0", "L < 1", "P_cols too large", "ldX < P_cols",
                 "y NULL", "slots beyond X without row_idx", "chop_sections", "max_sweeps",
                 "tol_move NaN"):
        h = Host(lib)
        dims_kw, ptr_kw, opts_kw = SHARED_CASES[case]
        _apply(h, dims_kw, opts_kw)
        assert f(*h.args(**ptr_kw), C.byref(h.d), None) == INVALID, case
    for case in ("lambdas NULL", "b_out NULL", "obj_out NULL", "group_threads", "work_order 2"):
        h = Host(lib)
        dims_kw, ptr_kw, opts_kw = FIT_CASES[case]
        _apply(h, dims_kw, opts_kw)
        assert f(*h.args(**ptr_kw), C.byref(h.d), None) == INVALID, case
    h = Host(lib)
    assert f(*h.args(), None, None) == INVALID
    # scratch beyond the fixed array: 2^22 slots of 8 columns
    h = Host(lib)
    h.d.total_rows = 1 << 22
    ri = np.zeros(1, np.int32)
    assert f(*h.args(row_idx=ri.ctypes.data), C.byref(h.d), None) == NOMEM


def test_empty_problem_sets_return_ok_without_work(lib):
    h = Host(lib, B=0, n=0)
    assert h.d.B == 0 and h.d.total_rows == 0
    args = h.args()
    for nm in ("ladlasso_fit_batched", "ladlasso_fit_batched_thread",
               "ladlasso_fit_batched_noalloc"):
        assert getattr(lib, nm)(*args, C.byref(h.d), None) == ll.OK, nm
    out = np.zeros(1, np.float32)
    assert lib.ladlasso_lambda_max(*args[:4], C.byref(h.d), out.ctypes.data, None) == ll.OK
    assert lib.ladlasso_lambda_path(out.ctypes.data, 0, 4, 0.5, out.ctypes.data, None) == ll.OK
    assert lib.ladlasso_path_loss(*args[:4], C.byref(h.d), h.b.ctypes.data, out.ctypes.data,
                                  None) == ll.OK
    assert _backward(lib, h) == ll.OK


def test_workspace_size_is_aligned_and_monotone(lib):
    f = lib.ladlasso_workspace_size
    rng = np.random.default_rng(0)
    for _ in range(200):
        B = int(rng.integers(0, 5000))
        P = int(rng.integers(1, KMAXP + 1))
        rows = int(rng.integers(0, 10 ** 7))
        L = int(rng.integers(1, 64))
        w = f(B, P, rows, L)
        assert w > 0 and w % 256 == 0, (B, P, rows, L, w)
        assert f(B + 1, P, rows, L) >= w
        assert f(B, P, rows + 1000, L) > w
        if P + 4 <= KMAXP:
            assert f(B, P + 4, rows, L) >= w
        assert f(B, P, rows, L + 1) == w  # the path length does not change it

"""ctypes binding of libladlasso.so (argument marshalling only).

Every step of the fit runs in the CUDA library; this module only turns torch
device tensors into pointers and sizes, allocates outputs and the workspace
with torch, and passes the current CUDA stream.  There is no CPU path: if the
library is not built, `lib()` raises.

Names follow include/ladlasso.h.  The batch layout ("problem set") is the
one documented there: X [rows_X, ldX] float32 row-major, y [total_rows],
row_idx [total_rows] int32 or None, offsets [B+1] int64, p [B] int32 or None.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libladlasso.so")
_lib = None

OK, ERR_INVALID, ERR_CUDA, ERR_NOMEM, ERR_WORKSPACE = 0, -1, -2, -3, -4
FIT_OK, FIT_MAX_ITERS, FIT_BAD_INPUT, FIT_NONUNIQUE = 0, 1, 2, 4


class Opts(C.Structure):
    """ladlasso_opts: the method's options (include/ladlasso.h); fill with
    default_opts(**overrides)."""
    _fields_ = [("tol_move", C.c_float), ("max_sweeps", C.c_int32), ("chop", C.c_int32),
                ("chop_bracket", C.c_float), ("chop_tol", C.c_float),
                ("chop_max_probes", C.c_int32), ("chop_max_extend", C.c_int32),
                ("probe_max_sweeps", C.c_int32), ("polish", C.c_int32),
                ("max_pivots", C.c_int32), ("tol_opt", C.c_float),
                ("lambda_min_floor", C.c_float), ("chop_sections", C.c_int32)]


class Dims(C.Structure):
    """ladlasso_dims: sizes and side arrays of one call; built by
    Problems.dims()."""
    _fields_ = [("B", C.c_int32), ("P_cols", C.c_int32), ("L", C.c_int32), ("n_max", C.c_int32),
                ("ldX", C.c_int64), ("rows_X", C.c_int64), ("total_rows", C.c_int64),
                ("p", C.c_void_p), ("n_rows", C.c_void_p), ("b_init", C.c_void_p), ("fit_status", C.c_void_p),
                ("basis_out", C.c_void_p), ("counters", C.c_void_p), ("workspace", C.c_void_p),
                ("workspace_bytes", C.c_size_t), ("opts", C.c_void_p),
                ("group_threads", C.c_int32), ("fits_per_block", C.c_int32),
                ("work_order", C.c_int32)]


class LadLassoError(RuntimeError):
    """A negative status from the library, or an argument the binding
    refuses before calling it."""


SYMBOLS = ["ladlasso_default_opts", "ladlasso_workspace_size", "ladlasso_lambda_max",
           "ladlasso_lambda_path", "ladlasso_fit_batched", "ladlasso_fit_batched_thread",
           "ladlasso_fit_backward", "ladlasso_status_string", "ladlasso_fit_batched_noalloc",
           "ladlasso_launch_shape", "ladlasso_path_loss"]


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise LadLassoError(f"{LIB_PATH} is not built; run paper_2510_15649_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    P, I32, I64, F = C.c_void_p, C.c_int32, C.c_int64, C.c_float
    DP = C.POINTER(Dims)
    L.ladlasso_default_opts.argtypes = [C.POINTER(Opts)]
    L.ladlasso_default_opts.restype = None
    L.ladlasso_workspace_size.argtypes = [I32, I32, I64, I32]
    L.ladlasso_workspace_size.restype = C.c_size_t
    L.ladlasso_lambda_max.argtypes = [P, P, P, P, DP, P, P]
    L.ladlasso_lambda_max.restype = C.c_int
    L.ladlasso_lambda_path.argtypes = [P, I32, I32, F, P, P]
    L.ladlasso_lambda_path.restype = C.c_int
    for nm in ("ladlasso_fit_batched", "ladlasso_fit_batched_thread",
               "ladlasso_fit_batched_noalloc"):
        fn = getattr(L, nm)
        fn.argtypes = [P, P, P, P, P, P, P, DP, P]
        fn.restype = C.c_int
    L.ladlasso_fit_backward.argtypes = [P, P, P, P, DP, I32, P, P, P, I64, P, P, P, I64, P,
                                        P, P, P, P, P, P, P, P]
    L.ladlasso_fit_backward.restype = C.c_int
    L.ladlasso_path_loss.argtypes = [P, P, P, P, DP, P, P, P]
    L.ladlasso_path_loss.restype = C.c_int
    L.ladlasso_launch_shape.argtypes = [DP, C.POINTER(I32), C.POINTER(I32), C.POINTER(I32)]
    L.ladlasso_launch_shape.restype = C.c_int
    L.ladlasso_status_string.argtypes = [C.c_int]
    L.ladlasso_status_string.restype = C.c_char_p
    _lib = L
    return L


def _check(rc: int):
    if rc != OK:
        raise LadLassoError(f"ladlasso: {lib().ladlasso_status_string(rc).decode()} ({rc})")


def default_opts(**kw) -> Opts:
    """The library's default options with the given fields overridden."""
    o = Opts()
    lib().ladlasso_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class _nvtx:
    """NVTX range around one library call (visible in profilers' timelines;
    a no-op where NVTX is unavailable)."""

    def __init__(self, name: str):
        self.name = name
        self.on = False

    def __enter__(self):
        try:
            torch.cuda.nvtx.range_push(self.name)
            self.on = True
        except Exception:
            pass
        return self

    def __exit__(self, *a):
        if self.on:
            torch.cuda.nvtx.range_pop()


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _need(t, name: str, dtype, dev, numel: int | None = None):
    """Raise unless tensor `t` (None allowed) is a contiguous `dtype` tensor
    on device `dev` with `numel` elements: the library reads raw pointers,
    so a host tensor, another dtype or a strided view would be misread."""
    if t is None:
        return
    if not isinstance(t, torch.Tensor):
        raise LadLassoError(f"{name} must be a torch tensor")
    if t.device != dev:
        raise LadLassoError(f"{name} is on {t.device}; the problem set is on {dev}")
    if t.dtype != dtype:
        raise LadLassoError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise LadLassoError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise LadLassoError(f"{name} has {t.numel()} elements, expected {numel}")


def _check_problems(pr: "Problems") -> None:
    """A problem set the library can read: CUDA tensors of the documented
    types (include/ladlasso.h), X row-major with at least P columns."""
    X = pr.X
    if not isinstance(X, torch.Tensor) or X.device.type != "cuda":
        raise LadLassoError("the problem set must be in CUDA device memory "
                            f"(X is on {getattr(X, 'device', type(X))})")
    _check_layout(pr)


def _check_layout(pr: "Problems") -> None:
    """Types, shapes and strides of a problem set, all on X's device."""
    X = pr.X
    dev = X.device
    if X.dtype != torch.float32 or X.dim() != 2:
        raise LadLassoError(f"X must be a 2-D float32 tensor, got {X.dtype} with {X.dim()} dims")
    if X.shape[1] < pr.P or (X.shape[0] > 0 and X.stride(1) != 1) or \
            (X.shape[0] > 1 and X.stride(0) < X.shape[1]):
        raise LadLassoError(f"X must be row-major with at least P = {pr.P} columns")
    _need(pr.y, "y", torch.float32, dev)
    if pr.y.dim() != 1:
        raise LadLassoError("y must be 1-D")
    _need(pr.offsets, "offsets", torch.int64, dev)
    if pr.offsets.numel() < 1:
        raise LadLassoError("offsets needs B + 1 >= 1 entries")
    _need(pr.row_idx, "row_idx", torch.int32, dev, int(pr.y.numel()))
    _need(pr.p, "p", torch.int32, dev, pr.B)
    _need(pr.n_rows, "n_rows", torch.int32, dev, pr.B)


_OUT_KINDS = {"b": (torch.float32, 3), "obj": (torch.float32, 1), "status": (torch.int32, 1),
              "basis": (torch.int32, 3), "counters": (torch.int32, 0)}


def _check_out(out: dict, B: int, L: int, P: int, dev, required=("b", "obj", "status")):
    """Result buffers handed to the library: b [B,L,P] and obj [B,L]
    float32, status [B,L], basis [B,L,P] and counters [B,L,8] int32."""
    for k in required:
        if k not in out:
            raise LadLassoError(f"out needs {k!r}")
    for k, t in out.items():
        if k in _OUT_KINDS:
            dtype, kind = _OUT_KINDS[k]
            per = P if kind == 3 else (8 if kind == 0 else 1)
            _need(t, f"out[{k!r}]", dtype, dev, B * L * per)


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


@dataclass
class Problems:
    """A problem set resident on the device (see include/ladlasso.h)."""
    X: torch.Tensor
    y: torch.Tensor
    offsets: torch.Tensor
    row_idx: torch.Tensor | None = None
    p: torch.Tensor | None = None
    P: int = 0
    n_max: int = 0
    n_rows: torch.Tensor | None = None

    @staticmethod
    def from_numpy(batch: dict, device="cuda") -> "Problems":
        """Upload a batch dict (synth layout) to `device`."""
        import numpy as np
        X = torch.as_tensor(np.ascontiguousarray(batch["X"], np.float32), device=device)
        y = torch.as_tensor(np.ascontiguousarray(batch["y"], np.float32), device=device)
        off = np.asarray(batch["offsets"], np.int64)
        offsets = torch.as_tensor(off, device=device)
        ri = batch.get("row_idx")
        row_idx = None if ri is None else torch.as_tensor(np.ascontiguousarray(ri, np.int32), device=device)
        p = torch.as_tensor(np.asarray(batch["p"], np.int32), device=device)
        n_max = int(np.max(np.diff(off))) if len(off) > 1 else 0
        return Problems(X=X, y=y, offsets=offsets, row_idx=row_idx, p=p,
                        P=int(X.shape[1]), n_max=n_max)

    @property
    def B(self) -> int:
        """Number of problems (offsets has B + 1 entries)."""
        return int(self.offsets.numel()) - 1

    def dims(self, L: int, workspace: torch.Tensor, opts: Opts | None = None, b_init=None,
             status=None, basis=None, counters=None) -> Dims:
        """ladlasso_dims for a call on this problem set with path length L,
        after checking every tensor the library will read."""
        _check_problems(self)
        d = Dims()
        d.B, d.P_cols, d.L, d.n_max = self.B, self.P, L, self.n_max
        d.ldX = int(self.X.stride(0))
        d.rows_X = int(self.X.shape[0])
        d.total_rows = int(self.y.numel())
        d.p = None if self.p is None else self.p.data_ptr()
        d.n_rows = None if self.n_rows is None else self.n_rows.data_ptr()
        d.b_init = None if b_init is None else b_init.data_ptr()
        d.fit_status = None if status is None else status.data_ptr()
        d.basis_out = None if basis is None else basis.data_ptr()
        d.counters = None if counters is None else counters.data_ptr()
        d.workspace = workspace.data_ptr()
        d.workspace_bytes = workspace.numel()
        d.opts = None if opts is None else C.addressof(opts)
        return d


def workspace_bytes(pr: Problems, L: int = 1) -> int:
    """Bytes of workspace the calls on `pr` need (ladlasso_workspace_size)."""
    n = lib().ladlasso_workspace_size(pr.B, pr.P, int(pr.y.numel()), L)
    if n == 0:
        raise LadLassoError("invalid sizes for workspace")
    return int(n)


def workspace(pr: Problems, L: int = 1) -> torch.Tensor:
    """Workspace buffer for `pr` (torch allocation, 256-byte aligned)."""
    n = workspace_bytes(pr, L)
    return torch.empty(n, dtype=torch.uint8, device=pr.X.device)


def lambda_max(pr: Problems, ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Per problem the smallest lambda at which b = 0 is optimal,
    max_j |x_j . sign(y)| over its rows and columns; NaN for a problem with
    bad input.  Returns [B] float32 on the device."""
    _check_problems(pr)
    ws = workspace(pr) if ws is None else ws
    _need(ws, "workspace", torch.uint8, pr.X.device)
    out = torch.empty(pr.B, dtype=torch.float32, device=pr.X.device)
    d = pr.dims(1, ws)
    with _nvtx("ladlasso_lambda_max"):
        _check(lib().ladlasso_lambda_max(_ptr(pr.X), _ptr(pr.y), _ptr(pr.row_idx),
                                         _ptr(pr.offsets), C.byref(d), _ptr(out), _stream(stream)))
    return out


def lambda_path(lmax: torch.Tensor, L: int, ratio: float = 1e-3, stream=None) -> torch.Tensor:
    """Geometric paths lmax[q] * ratio^(l / (L - 1)), l = 0..L-1 (lmax alone
    when L = 1).  Returns [B, L] float32 on the device."""
    B = int(lmax.numel())
    if lmax.device.type != "cuda":
        raise LadLassoError(f"lmax must be in CUDA device memory (it is on {lmax.device})")
    lmax = lmax.contiguous()
    _need(lmax, "lmax", torch.float32, lmax.device)
    out = torch.empty((B, L), dtype=torch.float32, device=lmax.device)
    _check(lib().ladlasso_lambda_path(_ptr(lmax), B, L, float(ratio), _ptr(out), _stream(stream)))
    return out


@dataclass(frozen=True)
class Launch:
    """Launch shape of the batched fit (ladlasso_dims.group_threads and
    .fits_per_block; zeros = the library's automatic choice)."""
    group_threads: int = 0
    fits_per_block: int = 0
    work_order: int = 0


def launch_shape(pr: Problems, launch: Launch | None = None) -> tuple:
    """(threads per fit, fits per block, max rows) the library would use."""
    d = Dims()
    d.P_cols, d.n_max = pr.P, pr.n_max
    if launch is not None:
        d.group_threads, d.fits_per_block = launch.group_threads, launch.fits_per_block
    g, f, m = C.c_int32(), C.c_int32(), C.c_int32()
    rc = lib().ladlasso_launch_shape(C.byref(d), C.byref(g), C.byref(f), C.byref(m))
    if rc not in (OK, ERR_NOMEM):
        _check(rc)
    return g.value, f.value, m.value


def fit(pr: Problems, lambdas: torch.Tensor, *, b_init=None, opts: Opts | None = None,
        basis: bool = False, counters: bool = False, per_thread: bool = False,
        ws: torch.Tensor | None = None, out: dict | None = None, stream=None,
        launch: Launch | None = None) -> dict:
    """Fit every problem along its lambda path.  lambdas: [B, L] float32 (device).
    `launch` overrides the launch shape (see tune.autotune).
    Returns dict(b [B,L,P], obj [B,L], status [B,L], basis?, counters?)."""
    _check_problems(pr)
    B, P = pr.B, pr.P
    lam = lambdas.reshape(B, -1).contiguous()
    L = int(lam.shape[1])
    dev = pr.X.device
    _need(lam, "lambdas", torch.float32, dev)
    _need(b_init, "b_init", torch.float32, dev, B * P)
    ws = workspace(pr, L) if ws is None else ws
    _need(ws, "workspace", torch.uint8, dev)
    if out is None:
        out = dict(b=torch.empty((B, L, P), dtype=torch.float32, device=dev),
                   obj=torch.empty((B, L), dtype=torch.float32, device=dev),
                   status=torch.empty((B, L), dtype=torch.int32, device=dev))
        if basis:
            out["basis"] = torch.empty((B, L, P), dtype=torch.int32, device=dev)
        if counters:
            out["counters"] = torch.empty((B, L, 8), dtype=torch.int32, device=dev)
    _check_out(out, B, L, P, dev)
    d = pr.dims(L, ws, opts, b_init=b_init, status=out["status"], basis=out.get("basis"),
                counters=out.get("counters"))
    if launch is not None:
        d.group_threads, d.fits_per_block = launch.group_threads, launch.fits_per_block
        d.work_order = launch.work_order
    fn = lib().ladlasso_fit_batched_thread if per_thread else lib().ladlasso_fit_batched
    with _nvtx("ladlasso_fit_batched_thread" if per_thread else "ladlasso_fit_batched"):
        _check(fn(_ptr(pr.X), _ptr(pr.y), _ptr(pr.row_idx), _ptr(pr.offsets), _ptr(lam),
                  _ptr(out["b"]), _ptr(out["obj"]), C.byref(d), _stream(stream)))
    return out


def path_loss(val: Problems, b: torch.Tensor, stream=None) -> torch.Tensor:
    """sum_v |y_v - x_v . b[q, l]| over the rows of problem q of `val`, for
    every path position l of b [B, L, P] (device).  Returns [B, L]."""
    _check_problems(val)
    B = val.B
    b = b.contiguous()
    if b.dim() != 3 or b.shape[0] != B or b.shape[2] != val.P:
        raise LadLassoError(f"b must be [B={B}, L, P={val.P}], got {tuple(b.shape)}")
    _need(b, "b", torch.float32, val.X.device)
    L = int(b.shape[1])
    out = torch.empty((B, L), dtype=torch.float32, device=val.X.device)
    d = val.dims(L, out)
    d.workspace, d.workspace_bytes = None, 0
    _check(lib().ladlasso_path_loss(_ptr(val.X), _ptr(val.y), _ptr(val.row_idx), _ptr(val.offsets),
                                    C.byref(d), _ptr(b.contiguous()), _ptr(out), _stream(stream)))
    return out


def fit_noalloc(pr: Problems, lambdas: torch.Tensor, *, opts: Opts | None = None,
                out: dict, stream=None) -> dict:
    """ladlasso_fit_batched_noalloc: the fit with the library's fixed
    scratch array instead of a workspace.  `out` holds preallocated
    b [B,L,P], obj [B,L], status [B,L] device tensors (nothing is allocated
    here either)."""
    _check_problems(pr)
    B = pr.B
    lam = lambdas.reshape(B, -1).contiguous()
    L = int(lam.shape[1])
    _need(lam, "lambdas", torch.float32, pr.X.device)
    _check_out(out, B, L, pr.P, pr.X.device)
    d = pr.dims(L, out["obj"], opts, status=out["status"])
    d.workspace = None
    d.workspace_bytes = 0
    _check(lib().ladlasso_fit_batched_noalloc(
        _ptr(pr.X), _ptr(pr.y), _ptr(pr.row_idx), _ptr(pr.offsets), _ptr(lam),
        _ptr(out["b"]), _ptr(out["obj"]), C.byref(d), _stream(stream)))
    return out


def fit_backward(pr: Problems, fwd: dict, pos: int, val: Problems, grad_up: torch.Tensor,
                 ws: torch.Tensor | None = None, opts: Opts | None = None, stream=None) -> dict:
    """Gradient of sum_v |y_v - x_v b| per problem at path position `pos`
    of a forward result that carries `basis`.  Returns dict(lam [B], y, X,
    yv, Xv, status [B], loss [B])."""
    _check_problems(pr)
    _check_problems(val)
    B, P = pr.B, pr.P
    if "basis" not in fwd:
        raise LadLassoError("the forward result needs its basis: fit(..., basis=True)")
    L = int(fwd["b"].shape[1])
    dev = pr.X.device
    if val.X.device != dev or val.X.shape[1] < P:
        raise LadLassoError(f"validation rows must be on {dev} with at least P = {P} columns")
    if not 0 <= pos < L:
        raise LadLassoError(f"path position {pos} outside 0..{L - 1}")
    _check_out(dict(b=fwd["b"], basis=fwd["basis"]), B, L, P, dev, required=("b", "basis"))
    ws = workspace(pr, L) if ws is None else ws
    _need(ws, "workspace", torch.uint8, dev)
    g = dict(lam=torch.empty(B, dtype=torch.float32, device=dev),
             y=torch.empty(pr.y.numel(), dtype=torch.float32, device=dev),
             X=torch.empty((pr.y.numel(), P), dtype=torch.float32, device=dev),
             yv=torch.empty(val.y.numel(), dtype=torch.float32, device=dev),
             Xv=torch.empty((val.y.numel(), P), dtype=torch.float32, device=dev),
             status=torch.empty(B, dtype=torch.int32, device=dev),
             loss=torch.empty(B, dtype=torch.float32, device=dev))
    d = pr.dims(L, ws, opts)
    up = grad_up.contiguous().float()
    _need(up, "grad_up", torch.float32, dev, B)
    with _nvtx("ladlasso_fit_backward"):
        _check(lib().ladlasso_fit_backward(
            _ptr(pr.X), _ptr(pr.y), _ptr(pr.row_idx), _ptr(pr.offsets), C.byref(d), int(pos),
            _ptr(fwd["b"]), _ptr(fwd["basis"]), _ptr(val.X), int(val.X.stride(0)), _ptr(val.y),
            _ptr(val.row_idx), _ptr(val.offsets), int(val.y.numel()), _ptr(up),
            _ptr(g["lam"]), _ptr(g["y"]), _ptr(g["X"]), _ptr(g["yv"]), _ptr(g["Xv"]),
            _ptr(g["status"]), _ptr(g["loss"]), _stream(stream)))
    return g


class ValidationLoss(torch.autograd.Function):
    """Per-problem validation LAD loss of the fit at one lambda, as a
    differentiable function of (training y, training X rows, lambda,
    validation y, validation X rows).

    forward(X, y, lam, Xv, yv, train, val): `train` / `val` are Problems
    whose X and y are the tensors X / y and Xv / yv; lam [B] is the lambda
    of each problem.  Returns loss [B].  Gradients flow to y, lam, yv and,
    per slot, to the X rows each problem uses (X must be indexed by slot:
    row_idx None).  The fit and both passes run in the CUDA library."""

    @staticmethod
    def forward(ctx, X, y, lam, Xv, yv, train: Problems, val: Problems, opts=None):
        fwd = fit(train, lam.reshape(-1, 1).contiguous(), basis=True, opts=opts)
        zero = torch.zeros(train.B, dtype=torch.float32, device=X.device)
        g = fit_backward(train, fwd, 0, val, zero)
        ctx.train, ctx.val, ctx.fwd = train, val, fwd
        ctx.mark_non_differentiable()
        return g["loss"]

    @staticmethod
    def backward(ctx, grad_loss):
        g = fit_backward(ctx.train, ctx.fwd, 0, ctx.val, grad_loss.contiguous())
        return g["X"], g["y"], g["lam"], g["Xv"], g["yv"], None, None, None

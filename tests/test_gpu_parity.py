"""Parity of the CUDA path (through the C ABI) with the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2510_15649_gb300 import synth

from gpu_common import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ll():
    import torch  # noqa: F401
    from paper_2510_15649_gb300 import build
    build.build()
    from paper_2510_15649_gb300 import ladlasso
    return ladlasso


def _run(ll, batch, lam_np, per_thread=False, n_max=None, **kw):
    import torch
    pr = ll.Problems.from_numpy(batch)
    if n_max is not None:
        pr.n_max = n_max
    lam = torch.as_tensor(np.asarray(lam_np, np.float32), device="cuda")
    out = ll.fit(pr, lam, per_thread=per_thread, basis=True, counters=True, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _oracle_lams(batch, L, ratio):
    B = len(batch["p"])
    lm = np.array([oracle.lambda_max(*oracle.problem(batch, q)) for q in range(B)])
    return (lm[:, None] * ratio ** (np.arange(L) / max(L - 1, 1))[None, :]).astype(np.float32)


@pytest.mark.parametrize("per_thread", [False, True])
def test_tiny_matches_brute_force(ll, per_thread):
    t = synth.tiny()
    batch = dict(X=t["X"], y=t["y"], row_idx=None, offsets=t["offsets"], p=t["p"])
    lam = np.array([[2.0]], np.float32)
    out = _run(ll, batch, lam, per_thread)
    fb, bb, _ = oracle.brute_force(t["X"].astype(float), t["y"].astype(float), 2.0)
    fg = oracle.objective(t["X"].astype(float), t["y"].astype(float), out["b"][0, 0].astype(float), 2.0)
    assert abs(fg - fb) / fb <= 1e-5
    assert np.array_equal(out["b"][0, 0] != 0, bb != 0)
    assert np.max(np.abs(out["b"][0, 0] - bb)) <= 1e-4 * max(1, np.abs(bb).max())
    assert out["status"][0, 0] == 0


@pytest.mark.parametrize("per_thread", [False, True])
def test_batched_small_parity(ll, per_thread):
    # several tiles of rows, ragged n, p from 1 to 12, a 5-point lambda path
    batch = synth.batched_like(48, 20, 700, 1, 12, R=800, P=12, seed=11)
    lam = _oracle_lams(batch, 5, 1e-3)
    out = _run(ll, batch, lam, per_thread)
    res = compare(batch, lam, out["b"], out["obj"], out["status"])
    assert not res["bad"], res["bad"][:10]
    assert np.all((out["status"] & 1) == 0)


@pytest.mark.parametrize("group", [64, 128, 512])
def test_batched_small_parity_multiwarp(ll, group):
    # the same problems with 2, 4 or 16 warps sharing each fit
    batch = synth.batched_like(48, 20, 700, 1, 12, R=800, P=12, seed=11)
    lam = _oracle_lams(batch, 5, 1e-3)
    out = _run(ll, batch, lam, launch=ll.Launch(group, 0, 0))
    res = compare(batch, lam, out["b"], out["obj"], out["status"])
    assert not res["bad"], res["bad"][:10]
    assert np.all((out["status"] & 1) == 0)
    assert res["support_checked"] >= 0.5 * res["checked"], res


def test_lambda_max_and_path(ll):
    import torch
    batch = synth.batched_like(40, 5, 500, 1, 16, R=600, P=16, seed=3)
    pr = ll.Problems.from_numpy(batch)
    lm = ll.lambda_max(pr)
    path = ll.lambda_path(lm, 6, 1e-3)
    torch.cuda.synchronize()
    lm = lm.cpu().numpy()
    for q in range(len(batch["p"])):
        ref = oracle.lambda_max(*oracle.problem(batch, q))
        assert abs(lm[q] - ref) <= 1e-5 * max(1, ref)
    p = path.cpu().numpy()
    np.testing.assert_allclose(p[:, 0], lm, rtol=1e-6)
    np.testing.assert_allclose(p[:, -1], lm * 1e-3, rtol=1e-5)


def test_block_and_thread_kernels_agree(ll):
    batch = synth.batched_like(24, 30, 400, 2, 10, R=500, P=10, seed=21)
    lam = _oracle_lams(batch, 3, 1e-2)
    a = _run(ll, batch, lam, False)
    b = _run(ll, batch, lam, True)
    fa = np.array([[oracle.objective(*oracle.problem(batch, q), a["b"][q, l, :batch["p"][q]].astype(float), lam[q, l])
                    for l in range(3)] for q in range(24)])
    fb = np.array([[oracle.objective(*oracle.problem(batch, q), b["b"][q, l, :batch["p"][q]].astype(float), lam[q, l])
                    for l in range(3)] for q in range(24)])
    assert np.max(np.abs(fa - fb) / np.maximum(1, fb)) <= 2e-5


def test_fit_is_identical_alone_and_in_a_batch(ll):
    batch = synth.batched_like(16, 30, 300, 2, 8, R=400, P=8, seed=5)
    lam = _oracle_lams(batch, 3, 1e-2)
    n_max = int(np.max(np.diff(batch["offsets"])))
    full = _run(ll, batch, lam)
    for q in [0, 7, 15]:
        o0, o1 = batch["offsets"][q], batch["offsets"][q + 1]
        one = dict(X=batch["X"], y=batch["y"][o0:o1], row_idx=batch["row_idx"][o0:o1],
                   offsets=np.array([0, o1 - o0], np.int64), p=batch["p"][q:q + 1])
        # same n_max so the same block shape is used
        alone = _run(ll, one, lam[q:q + 1], n_max=n_max)
        np.testing.assert_array_equal(alone["b"][0], full["b"][q])
        np.testing.assert_array_equal(alone["obj"][0], full["obj"][q])


def test_edge_cases(ll):
    import torch
    # empty problem, p = 1, a NaN lambda, a negative lambda
    X = np.random.default_rng(0).standard_normal((50, 3)).astype(np.float32)
    y = (X @ np.array([1.0, -2, 0]) + 0.1).astype(np.float32)
    batch = dict(X=X, y=y[:45], row_idx=np.arange(45, dtype=np.int32),
                 offsets=np.array([0, 0, 20, 45], np.int64), p=np.array([3, 1, 3], np.int32))
    lam = np.array([[1.0, 0.5], [1.0, np.nan], [-1.0, 0.1]], np.float32)
    out = _run(ll, batch, lam)
    assert np.all(out["b"][0] == 0) and np.all(out["status"][0] == 0)
    assert out["status"][1, 1] == 2 and out["status"][2, 0] == 2
    assert np.all(out["b"][1, 1] == 0)
    res = compare(batch, lam, out["b"], out["obj"], out["status"], problems=[1])
    assert not [b for b in res["bad"] if b[1] == 0], res["bad"]
    # row index out of range -> BAD_INPUT for that problem only
    bad = dict(batch)
    ri = batch["row_idx"].copy()
    ri[30] = 10_000
    bad["row_idx"] = ri
    out = _run(ll, bad, lam)
    assert np.all(out["status"][2] == 2) and np.all(out["b"][2] == 0)
    assert out["status"][1, 0] != 2
    # non-monotone offsets -> every problem BAD_INPUT
    nm = dict(batch)
    nm["offsets"] = np.array([0, 25, 20, 45], np.int64)
    out = _run(ll, nm, lam)
    assert np.all(out["status"] == 2)


def test_invalid_arguments_return_errors(ll):
    import ctypes as C
    import torch
    L = ll.lib()
    d = ll.Dims()
    d.B, d.P_cols, d.L, d.n_max = 1, 4, 1, 10
    d.ldX, d.rows_X, d.total_rows = 4, 10, 10
    x = torch.zeros(64, device="cuda")
    off = torch.tensor([0, 10], dtype=torch.int64, device="cuda")
    p = C.c_void_p(x.data_ptr())
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    # no workspace
    assert L.ladlasso_fit_batched(p, p, None, C.c_void_p(off.data_ptr()), p, p, p, C.byref(d), s) == ll.ERR_WORKSPACE
    d.P_cols = 0
    assert L.ladlasso_fit_batched(p, p, None, C.c_void_p(off.data_ptr()), p, p, p, C.byref(d), s) == ll.ERR_INVALID
    assert L.ladlasso_lambda_path(p, 1, 1, 2.0, p, s) == ll.ERR_INVALID


@pytest.mark.parametrize("per_thread", [False, True])
def test_four_section_chop_parity(ll, per_thread):
    # the "quadrature" reading of the chop (three inner probes per step)
    batch = synth.batched_like(32, 20, 600, 2, 10, R=700, P=10, seed=13)
    lam = _oracle_lams(batch, 4, 1e-3)
    out = _run(ll, batch, lam, per_thread, opts=ll.default_opts(chop_sections=4))
    res = compare(batch, lam, out["b"], out["obj"], out["status"],
                  opts=oracle.default_opts(chop_sections=4))
    assert not res["bad"], res["bad"][:10]
    # the chop ran and probed in threes
    c = out["counters"]
    ran = (c[..., 3] & 2) != 0
    assert ran.any()


def test_iteration_caps_report_max_iters_and_keep_the_best_point(ll):
    # one CCD sweep and one polish pivot: fits that needed more are flagged
    # MAX_ITERS; their objective is never above the starting point's
    batch = synth.batched_like(24, 100, 400, 4, 10, R=500, P=10, seed=17)
    lam = _oracle_lams(batch, 2, 1e-2)
    capped = _run(ll, batch, lam, opts=ll.default_opts(max_sweeps=1, max_pivots=1, chop=0))
    full = _run(ll, batch, lam)
    st = capped["status"]
    assert np.mean((st & 1) != 0) > 0.5
    assert np.all((st & 2) == 0)
    lh = lam.astype(np.float64)
    for q in range(24):
        X, y = oracle.problem(batch, q)
        p = X.shape[1]
        f0 = oracle.objective(X, y, np.zeros(p), lh[q, 0])
        fc = oracle.objective(X, y, capped["b"][q, 0, :p].astype(np.float64), lh[q, 0])
        ff = oracle.objective(X, y, full["b"][q, 0, :p].astype(np.float64), lh[q, 0])
        assert fc <= f0 * (1 + 1e-6) and ff <= fc * (1 + 1e-6)

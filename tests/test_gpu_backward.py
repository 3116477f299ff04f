"""Adjoint kernel (ladlasso_fit_backward) against the FP64 oracle's
active-set gradient of the validation LAD loss, and the autograd wrapper.
The oracle gradient itself is pinned to central finite differences in
tests/test_oracle.py."""
import numpy as np
import pytest

import oracle
from gpu_common import well_separated
from paper_2510_15649_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ll():
    from paper_2510_15649_gb300 import build
    build.build()
    from paper_2510_15649_gb300 import ladlasso
    return ladlasso


def _setup(ll, B=24, n=140, ntr=110, p=6, seed=3):
    import torch
    d = synth.diff(B=B, n=n, n_train=ntr, p=p, seed=seed)
    tr, va = d["train"], d["val"]
    lam = np.array([0.1 * oracle.lambda_max(*oracle.problem(tr, q)) for q in range(B)], np.float32)
    ptr = ll.Problems.from_numpy(tr)
    pva = ll.Problems.from_numpy(va)
    return d, tr, va, lam, ptr, pva


def test_backward_matches_oracle_active_set_gradient(ll):
    import torch
    d, tr, va, lam, ptr, pva = _setup(ll)
    B = len(lam)
    lam_t = torch.as_tensor(lam, device="cuda").reshape(B, 1)
    fwd = ll.fit(ptr, lam_t, basis=True)
    up = torch.linspace(0.5, 2.0, B, device="cuda")
    g = ll.fit_backward(ptr, fwd, 0, pva, up)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in g.items()}
    checked = _check_against_oracle(g, fwd["b"].cpu().numpy()[:, 0], lam, up.cpu().numpy(),
                                    tr, va, range(B))
    assert checked >= B // 2


def test_backward_full_size_sampled(ll):
    # the differentiation workload as the benchmark runs it: 512 problems of
    # 400 training and 100 validation rows, 16 columns, lambda = 0.1 lambda_max
    # of the training rows (computed on the GPU); 32 problems compared
    import torch
    d = synth.diff()
    tr, va = d["train"], d["val"]
    ptr, pva = ll.Problems.from_numpy(tr), ll.Problems.from_numpy(va)
    B = ptr.B
    assert B == 512 and ptr.P == 16
    lam_t = (0.1 * ll.lambda_max(ptr)).reshape(B, 1).contiguous()
    fwd = ll.fit(ptr, lam_t, basis=True)
    up = torch.ones(B, device="cuda")
    g = ll.fit_backward(ptr, fwd, 0, pva, up)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in g.items()}
    qs = range(0, B, 16)
    checked = _check_against_oracle(g, fwd["b"].cpu().numpy()[:, 0], lam_t.cpu().numpy()[:, 0],
                                    up.cpu().numpy(), tr, va, qs, separated_only=True)
    assert checked >= len(qs) // 2


def _well_separated(X, y, ref, lam):
    """The parity bar's uniqueness test (tests/gpu_common.py): a strict
    vertex whose multipliers keep more slack than float32 can misjudge and
    whose support is the same at lambda * (1 -+ LAM_REL), so float32 cannot
    land on another vertex."""
    return well_separated(X, y, ref["b"][0], ref["basis"][0], lam)


def _check_against_oracle(g, bg, lam, upn, tr, va, qs, separated_only=False):
    """Per sampled problem: the validation loss at the GPU's coefficients,
    and, where both sides end at a strict vertex (well separated from its
    neighbours at float32 resolution when `separated_only`), every gradient
    entry within 1e-3 max(1, |g|) of the oracle's active-set gradient and a
    zero lambda derivative.  Returns how many problems had their gradient
    checked."""
    checked = 0
    for q in qs:
        X, y = oracle.problem(tr, q)
        Xv, yv = oracle.problem(va, q)
        o0, o1 = tr["offsets"][q], tr["offsets"][q + 1]
        v0, v1 = va["offsets"][q], va["offsets"][q + 1]
        ref = oracle.fit_path(X, y, [float(lam[q])])
        # validation loss at the GPU's own coefficients
        lv = np.abs(yv - Xv @ bg[q].astype(np.float64)).sum()
        assert abs(g["loss"][q] - lv) <= 1e-5 * max(1.0, lv)
        if ref["status"][0] != oracle.FIT_OK or g["status"][q] != 0:
            continue  # not a strict vertex: the gradient is not defined there
        if separated_only and not _well_separated(X, y, ref, float(lam[q])):
            continue
        og = oracle.grad(X, y, ref["b"][0], ref["basis"][0], Xv, yv, up=float(upn[q]))
        assert og["ok"]
        tol = lambda a: 1e-3 * np.maximum(1.0, np.abs(a))
        assert np.all(np.abs(g["y"][o0:o1] - og["gy"]) <= tol(og["gy"]))
        assert np.all(np.abs(g["X"][o0:o1] - og["gX"]) <= tol(og["gX"]))
        assert np.all(np.abs(g["yv"][v0:v1] - og["gyv"]) <= tol(og["gyv"]))
        assert np.all(np.abs(g["Xv"][v0:v1] - og["gXv"]) <= tol(og["gXv"]))
        assert g["lam"][q] == 0.0
        checked += 1
    return checked


def test_autograd_function_matches_backward_entry_point(ll):
    import torch
    d, tr, va, lam, ptr, pva = _setup(ll, B=8, seed=4)
    B = len(lam)
    X = ptr.X.clone().requires_grad_(True)
    y = ptr.y.clone().requires_grad_(True)
    Xv = pva.X.clone().requires_grad_(True)
    yv = pva.y.clone().requires_grad_(True)
    lam_t = torch.as_tensor(lam, device="cuda").requires_grad_(True)
    train = ll.Problems(X=X.detach(), y=y.detach(), offsets=ptr.offsets, p=ptr.p, P=ptr.P,
                        n_max=ptr.n_max)
    val = ll.Problems(X=Xv.detach(), y=yv.detach(), offsets=pva.offsets, p=pva.p, P=pva.P,
                      n_max=pva.n_max)
    loss = ll.ValidationLoss.apply(X, y, lam_t, Xv, yv, train, val)
    w = torch.arange(1, B + 1, dtype=torch.float32, device="cuda")
    (loss * w).sum().backward()
    fwd = ll.fit(train, lam_t.detach().reshape(B, 1), basis=True)
    g = ll.fit_backward(train, fwd, 0, val, w)
    torch.cuda.synchronize()
    np.testing.assert_allclose(y.grad.cpu().numpy(), g["y"].cpu().numpy(), rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(X.grad.cpu().numpy(), g["X"].cpu().numpy(), rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(yv.grad.cpu().numpy(), g["yv"].cpu().numpy(), rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(lam_t.grad.cpu().numpy(), g["lam"].cpu().numpy())

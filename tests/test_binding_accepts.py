"""The binding's tensor checks accept every problem set and result buffer
the package itself builds (on CPU tensors here: the layout checks do not
depend on the device), so a valid call is never refused: the upload of each
input recipe, the serving pool and its admission sets, cross-validation's
split sets, the autotuner's sample sets, and the buffers fit() allocates."""
import numpy as np
import torch

from paper_2510_15649_gb300 import cv, synth, tune
from paper_2510_15649_gb300 import ladlasso as ll
from paper_2510_15649_gb300.serve import Server, admission_offsets


def _ok(pr):
    ll._check_layout(pr)


def test_uploaded_recipes_pass():
    for b in (synth.batched_like(20, 5, 60, 1, 8, R=80, P=8, seed=1),
              synth.large(B=2, n=300, p=12),
              synth.diff(B=3)["train"], synth.diff(B=3)["val"],
              synth.tiny()):
        _ok(ll.Problems.from_numpy(b, device="cpu"))


def test_serving_pool_and_admission_sets_pass():
    srv = Server(slots=6, cap=50, P=8, L=2, device="cpu")
    _ok(srv.pr)
    srv.h_n[[1, 4]] = [20, 35]
    srv.h_p[[1, 4]] = [3, 8]
    ss = np.array([1, 4], np.int64)
    sub = ll.Problems(X=srv.X, y=srv.y, offsets=torch.from_numpy(admission_offsets(ss, 50, 6)),
                      p=torch.from_numpy(srv.h_p[ss]), P=8, n_max=50,
                      n_rows=torch.from_numpy(srv.h_n[ss]))
    _ok(sub)
    # a launch takes up to K path positions per slot, warm-started from b_state
    ll._check_out(dict(b=srv.b, obj=srv.obj, status=srv.status), srv.S, srv.K, 8, srv.X.device)
    assert srv.K == 2 and srv.lam_step.shape == (srv.S, srv.K)
    assert srv.b_state.numel() == srv.S * srv.P


def test_cross_validation_sets_pass():
    rng = np.random.default_rng(2)
    X = torch.as_tensor(rng.standard_normal((40, 5)).astype(np.float32))
    y = torch.as_tensor(rng.standard_normal(40).astype(np.float32))
    sp = cv.kfold_splits(40, 4, seed=1)
    tr = cv._problem_set(X, [y[torch.as_tensor(t)] for t, _ in sp], [t for t, _ in sp], 5, 5)
    ho = cv._problem_set(X, [y[torch.as_tensor(h)] for _, h in sp], [h for _, h in sp], 5, 5)
    _ok(tr)
    _ok(ho)


def test_autotuner_sample_sets_pass():
    b = synth.batched_like(12, 5, 40, 2, 6, R=60, P=6, seed=4)
    pr = ll.Problems.from_numpy(b, device="cpu")
    lam = torch.ones((pr.B, 3))
    sub, sl = tune._subset(pr, lam, 3)
    _ok(sub)
    assert sl.is_contiguous() and sl.dtype == torch.float32


def test_buffers_fit_allocates_pass():
    B, L, P = 7, 4, 6
    dev = torch.device("cpu")
    out = dict(b=torch.empty((B, L, P), dtype=torch.float32, device=dev),
               obj=torch.empty((B, L), dtype=torch.float32, device=dev),
               status=torch.empty((B, L), dtype=torch.int32, device=dev),
               basis=torch.empty((B, L, P), dtype=torch.int32, device=dev),
               counters=torch.empty((B, L, 8), dtype=torch.int32, device=dev))
    ll._check_out(out, B, L, P, dev)

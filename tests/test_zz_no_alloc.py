"""ladlasso_fit_batched_noalloc against ladlasso_fit_batched.

The no-allocation entry point serves callers that cannot allocate device
memory while they fit (a plugin whose host framework owns every device
allocation, a serving loop that must not call cudaMalloc once running).  It
runs the same block-per-fit kernel with the library's fixed scratch array in
place of a caller workspace, so its results must match the workspace entry
point's within the parity tolerance -- on two calls in a row, since the
array keeps the previous call's contents.  This file sorts last so that a
run stopping at the first failure has run every other test before it.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2510_15649_gb300 import synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_workspace_entry_point_twice():
    import torch
    from paper_2510_15649_gb300 import build
    build.build()
    from paper_2510_15649_gb300 import ladlasso as ll

    batch = synth.batched_like(40, 30, 600, 2, 12, R=700, P=12, seed=17)
    pr = ll.Problems.from_numpy(batch)
    lmax = ll.lambda_max(pr)
    lam = ll.lambda_path(lmax, 4, 1e-3)
    ref = ll.fit(pr, lam)
    B, L, P = pr.B, 4, pr.P
    outs = []
    for _ in range(2):
        out = dict(b=torch.full((B, L, P), 7.0, device="cuda"),
                   obj=torch.full((B, L), -1.0, device="cuda"),
                   status=torch.full((B, L), 99, dtype=torch.int32, device="cuda"))
        ll.fit_noalloc(pr, lam, out=out)
        torch.cuda.synchronize()
        outs.append({k: v.cpu().numpy() for k, v in out.items()})
    r = {k: v.cpu().numpy() for k, v in ref.items()}
    for o in outs:
        np.testing.assert_array_equal(o["status"], r["status"])
        rel = np.abs(o["obj"] - r["obj"]) / np.maximum(1.0, np.abs(r["obj"]))
        assert rel.max() <= 1e-5
        scale = np.maximum(1.0, np.abs(r["b"]).max(axis=2, keepdims=True))
        assert (np.abs(o["b"] - r["b"]) / scale).max() <= 1e-4


def test_noalloc_rejects_problem_sets_beyond_its_array():
    import torch
    from paper_2510_15649_gb300 import ladlasso as ll
    L = ll.lib()
    d = ll.Dims()
    # 2 million slots x 8 columns of float32 = 64 MB > the 32 MiB array
    d.B, d.P_cols, d.L, d.n_max = 1, 8, 1, 2_000_000
    d.ldX, d.rows_X, d.total_rows = 8, 2_000_000, 2_000_000
    x = torch.zeros(16, device="cuda")
    off = torch.tensor([0, 2_000_000], dtype=torch.int64, device="cuda")
    p = C.c_void_p(x.data_ptr())
    rc = L.ladlasso_fit_batched_noalloc(p, p, None, C.c_void_p(off.data_ptr()), p, p, p,
                                        C.byref(d), None)
    assert rc == ll.ERR_NOMEM

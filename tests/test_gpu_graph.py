"""The batched fit captured in a CUDA graph replays with results identical
to the eager call (the library makes no allocation and no synchronisation
inside a call; its one-time launch attributes are set outside capture by a
first eager call)."""
import numpy as np
import pytest

from paper_2510_15649_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ll():
    import torch  # noqa: F401
    from paper_2510_15649_gb300 import build
    build.build()
    from paper_2510_15649_gb300 import ladlasso
    return ladlasso


def test_captured_step_replays_identically(ll):
    import torch
    batch = synth.batched_like(64, 30, 800, 2, 16, R=900, P=16, seed=61)
    pr = ll.Problems.from_numpy(batch)
    L = 4
    ws = ll.workspace(pr, L)
    dev = pr.X.device
    out = dict(b=torch.empty((pr.B, L, pr.P), device=dev), obj=torch.empty((pr.B, L), device=dev),
               status=torch.empty((pr.B, L), dtype=torch.int32, device=dev))
    lmax = torch.empty(pr.B, device=dev)
    lam = torch.empty((pr.B, L), device=dev)

    def step():
        lmax.copy_(ll.lambda_max(pr, ws))
        lam.copy_(ll.lambda_path(lmax, L, 1e-3))
        ll.fit(pr, lam, ws=ws, out=out)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()  # eager: sets kernel attributes, warms up
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    ref = {k: v.clone() for k, v in out.items()}
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        step()
    for _ in range(2):
        for v in out.values():
            v.zero_()
        g.replay()
        torch.cuda.synchronize()
        for k in ref:
            assert torch.equal(out[k], ref[k]), k
    assert np.all((ref["status"].cpu().numpy() & 2) == 0)

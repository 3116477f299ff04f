"""The Python binding refuses tensors the library would misread (host
memory, other dtypes, strided views, wrong sizes) with an error before any
library call; the checks read tensor metadata only (no GPU needed)."""
import numpy as np
import pytest
import torch

from paper_2510_15649_gb300 import ladlasso as ll
from paper_2510_15649_gb300 import synth


def _cpu_problems():
    b = synth.batched_like(5, 10, 40, 2, 6, R=60, P=6, seed=9)
    return ll.Problems.from_numpy(b, device="cpu")


def test_host_problem_sets_are_refused_by_every_entry_point():
    pr = _cpu_problems()
    lam = torch.ones((pr.B, 2))
    with pytest.raises(ll.LadLassoError, match="CUDA device memory"):
        ll.fit(pr, lam)
    with pytest.raises(ll.LadLassoError, match="CUDA device memory"):
        ll.lambda_max(pr)
    with pytest.raises(ll.LadLassoError, match="CUDA device memory"):
        ll.path_loss(pr, torch.zeros((pr.B, 2, pr.P)))
    with pytest.raises(ll.LadLassoError, match="CUDA device memory"):
        ll.fit_noalloc(pr, lam, out={})
    with pytest.raises(ll.LadLassoError, match="CUDA device memory"):
        ll.fit_backward(pr, dict(b=torch.zeros((pr.B, 1, pr.P))), 0, pr, torch.ones(pr.B))
    with pytest.raises(ll.LadLassoError, match="CUDA device memory"):
        ll.lambda_path(torch.ones(3), 4)


def _broken(**kw):
    pr = _cpu_problems()
    for k, v in kw.items():
        setattr(pr, k, v)
    return pr


@pytest.mark.parametrize("case", [
    "X float64", "X transposed", "X every other column", "X narrower than P", "X 1-D",
    "y float64", "y 2-D",
    "y strided", "offsets int32", "offsets empty", "row_idx int64", "row_idx short",
    "p wrong count", "p int64", "n_rows float", "y on another device"])
def test_layout_errors(case):
    pr = _cpu_problems()
    X, y = pr.X, pr.y
    bad = {
        "X float64": dict(X=X.double()),
        "X transposed": dict(X=X.t().contiguous().t()),
        # rows far enough apart, but the columns are not adjacent
        "X every other column": dict(X=torch.zeros((X.shape[0], 2 * X.shape[1]))[:, ::2]),
        "X narrower than P": dict(X=X[:, :4].contiguous()),
        "X 1-D": dict(X=X.reshape(-1)),
        "y float64": dict(y=y.double()),
        "y 2-D": dict(y=y.reshape(-1, 1)),
        "y strided": dict(y=torch.stack([y, y], 1)[:, 0]),
        "offsets int32": dict(offsets=pr.offsets.int()),
        "offsets empty": dict(offsets=pr.offsets[:0]),
        "row_idx int64": dict(row_idx=pr.row_idx.long()),
        "row_idx short": dict(row_idx=pr.row_idx[:-1]),
        "p wrong count": dict(p=pr.p[:-1]),
        "p int64": dict(p=pr.p.long()),
        "n_rows float": dict(n_rows=torch.ones(pr.B)),
        "y on another device": dict(y=y.to("meta")),
    }[case]
    with pytest.raises(ll.LadLassoError):
        ll._check_layout(_broken(**bad))


def test_valid_layouts_pass():
    pr = _cpu_problems()
    ll._check_layout(pr)
    # a row-major view with a longer row stride (ldX > P) is accepted
    wide = torch.zeros((pr.X.shape[0], 10))
    wide[:, :6] = pr.X
    ll._check_layout(_broken(X=wide[:, :8]))
    ll._check_layout(_broken(row_idx=None, X=torch.zeros((int(pr.y.numel()), 6))))
    ll._check_layout(_broken(n_rows=torch.ones(pr.B, dtype=torch.int32)))


def test_result_buffers_are_checked():
    dev = torch.device("cpu")
    B, L, P = 3, 2, 4
    good = dict(b=torch.zeros((B, L, P)), obj=torch.zeros((B, L)),
                status=torch.zeros((B, L), dtype=torch.int32),
                basis=torch.zeros((B, L, P), dtype=torch.int32),
                counters=torch.zeros((B, L, 8), dtype=torch.int32))
    ll._check_out(good, B, L, P, dev)
    for k, v in [("b", torch.zeros((B, L, P + 1))), ("obj", torch.zeros((B, L), dtype=torch.float64)),
                 ("status", torch.zeros((B, L))), ("basis", torch.zeros((B, L, P), dtype=torch.int32)[:, :1]),
                 ("counters", torch.zeros((B, L, 7), dtype=torch.int32)),
                 ("b", torch.zeros((B, P, L)).transpose(1, 2))]:
        with pytest.raises(ll.LadLassoError):
            ll._check_out({**good, k: v}, B, L, P, dev)
    with pytest.raises(ll.LadLassoError, match="needs 'status'"):
        ll._check_out(dict(b=good["b"], obj=good["obj"]), B, L, P, dev)
    ll._check_out(dict(b=good["b"], basis=good["basis"]), B, L, P, dev, required=("b", "basis"))
    assert np.all(good["b"].numpy() == 0)


def test_missing_library_fails_loudly(monkeypatch):
    # no CPU fallback: without the built library every call raises
    monkeypatch.setattr(ll, "_lib", None)
    monkeypatch.setattr(ll, "LIB_PATH", ll.LIB_PATH + ".missing")
    with pytest.raises(ll.LadLassoError, match="not built"):
        ll.lib()
    with pytest.raises(ll.LadLassoError, match="not built"):
        ll.default_opts()

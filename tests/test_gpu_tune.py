"""Launch shapes and the autotuner: results do not depend on the number of
fits per block; the block-per-fit shape agrees with the one-warp shape
within the parity tolerance; the autotuner returns one of the candidates."""
import numpy as np
import pytest

import oracle
from paper_2510_15649_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ll():
    import torch  # noqa: F401
    from paper_2510_15649_gb300 import build
    build.build()
    from paper_2510_15649_gb300 import ladlasso
    return ladlasso


def _setup(ll):
    import torch
    batch = synth.batched_like(96, 30, 900, 2, 16, R=1000, P=16, seed=41)
    pr = ll.Problems.from_numpy(batch)
    lam = ll.lambda_path(ll.lambda_max(pr), 4, 1e-2)
    torch.cuda.synchronize()
    return batch, pr, lam


def test_results_do_not_depend_on_fits_per_block(ll):
    import torch
    batch, pr, lam = _setup(ll)
    ref = ll.fit(pr, lam)
    for f in (1, 3):
        out = ll.fit(pr, lam, launch=ll.Launch(32, f))
        torch.cuda.synchronize()
        assert torch.equal(out["b"], ref["b"]) and torch.equal(out["obj"], ref["obj"])
        assert torch.equal(out["status"], ref["status"])


def test_block_shape_agrees_with_warp_shape(ll):
    import torch
    batch, pr, lam = _setup(ll)
    a = ll.fit(pr, lam, launch=ll.Launch(32, 0))
    b = ll.fit(pr, lam, launch=ll.Launch(512, 0))
    torch.cuda.synchronize()
    lh = lam.cpu().numpy().astype(np.float64)
    ba, bb = a["b"].cpu().numpy(), b["b"].cpu().numpy()
    for q in range(0, 96, 7):
        X, y = oracle.problem(batch, q)
        p = X.shape[1]
        for l in range(4):
            fa = oracle.objective(X, y, ba[q, l, :p].astype(np.float64), lh[q, l])
            fb = oracle.objective(X, y, bb[q, l, :p].astype(np.float64), lh[q, l])
            assert abs(fa - fb) <= 1e-5 * max(1.0, fa), (q, l, fa, fb)


def test_autotune_picks_a_candidate_and_caches(ll):
    from paper_2510_15649_gb300 import tune
    batch, pr, lam = _setup(ll)
    cands = tune.candidates(pr)
    assert ll.Launch(512, 0) in cands and any(c.group_threads == 32 for c in cands)
    choice, times = tune.autotune(pr, lam, sample_problems=32)
    assert choice in cands and set(times) == set(cands)
    assert all(t > 0 for t in times.values())
    again, _ = tune.autotune(pr, lam, sample_problems=32)
    assert again == choice


def test_results_do_not_depend_on_work_order(ll):
    import torch
    batch, pr, lam = _setup(ll)
    a = ll.fit(pr, lam, launch=ll.Launch(32, 0, 0))
    b = ll.fit(pr, lam, launch=ll.Launch(32, 0, 1))
    torch.cuda.synchronize()
    assert torch.equal(a["b"], b["b"]) and torch.equal(a["obj"], b["obj"])


def permute_problems(batch, perm):
    """The batch with its problems in the order `perm` (rows and targets
    move with their problem; the shared design is unchanged)."""
    off = batch["offsets"]
    rows = [batch["row_idx"][off[q]:off[q + 1]] for q in perm]
    ys = [batch["y"][off[q]:off[q + 1]] for q in perm]
    lens = np.array([len(r) for r in rows], np.int64)
    return dict(X=batch["X"], y=np.concatenate(ys), row_idx=np.concatenate(rows),
                offsets=np.concatenate([[0], np.cumsum(lens)]).astype(np.int64),
                p=np.asarray(batch["p"])[perm])


def test_results_do_not_depend_on_problem_order(ll):
    # each fit is one warp's own arithmetic: reordering the problems of a
    # batch (same n_max, so the same launch shape) moves the results with
    # them, bit for bit
    import torch
    batch, pr, lam = _setup(ll)
    perm = np.random.default_rng(3).permutation(pr.B)
    pb = permute_problems(batch, perm)
    prp = ll.Problems.from_numpy(pb)
    assert prp.n_max == pr.n_max
    a = ll.fit(pr, lam)
    b = ll.fit(prp, lam[torch.as_tensor(perm, device=lam.device)].contiguous())
    torch.cuda.synchronize()
    for k in ("b", "obj", "status"):
        assert np.array_equal(a[k].cpu().numpy()[perm], b[k].cpu().numpy()), k

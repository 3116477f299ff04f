"""Host logic of the autotuner: candidate launch shapes (no GPU: the
library's launch_shape entry point touches no device)."""
from paper_2510_15649_gb300 import ladlasso as ll
from paper_2510_15649_gb300 import tune


class Pr:  # the fields candidates() reads
    def __init__(self, P, n_max):
        self.P, self.n_max = P, n_max


def test_candidates_cover_every_shape_and_order_when_all_fit():
    c = tune.candidates(Pr(32, 2000))
    for gt in (32, 64, 128):
        grp = [x for x in c if x.group_threads == gt]
        _, fmax, _ = ll.launch_shape(Pr(32, 2000), ll.Launch(gt, 0))
        assert fmax >= 1 and fmax * gt <= 512
        assert {x.fits_per_block for x in grp} == set(range(max(1, fmax // 3), fmax + 1))
        assert {x.work_order for x in grp} == {0, 1}
    block = [x for x in c if x.group_threads == 512]
    assert block == [ll.Launch(512, 0, 0), ll.Launch(512, 0, 1)]
    assert len(set(c)) == len(c)


def test_long_problems_only_get_the_block_shape():
    c = tune.candidates(Pr(128, 20000))
    assert c and all(x.group_threads == 512 for x in c)


def test_no_candidate_beyond_every_shape():
    assert tune.candidates(Pr(128, 10 ** 6)) == []


def _cpu_problems(B=6, seed=2):
    from paper_2510_15649_gb300 import synth
    return ll.Problems.from_numpy(synth.batched_like(B, 5, 30, 2, 6, R=60, P=6, seed=seed),
                                  device="cpu")


def test_cache_round_trips_through_json():
    import os
    tune._cache.clear()
    key = tune.cache_key(_cpu_problems(), 16, None, "GB300")
    times = {ll.Launch(32, 3, 0): 1.046, ll.Launch(32, 5, 1): 1.107, ll.Launch(512, 0, 0): 2.0}
    tune._cache[key] = (ll.Launch(32, 3, 0), times)
    d = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_build")
    os.makedirs(d, exist_ok=True)
    path = os.path.join(d, f"tune_cache_test_{os.getpid()}.json")
    try:
        tune.save_cache(path)
        tune._cache.clear()
        assert tune.load_cache(path) == 1
    finally:
        os.remove(path)
    choice, t2 = tune._cache[key]
    assert choice == ll.Launch(32, 3, 0) and t2 == times
    tune._cache.clear()


def test_cache_key_tells_problem_sets_and_options_apart():
    a, b = _cpu_problems(seed=2), _cpu_problems(seed=3)
    assert int(a.y.numel()) != int(b.y.numel())
    assert tune.cache_key(a, 4) == tune.cache_key(a, 4, ll.default_opts())
    assert tune.cache_key(a, 4) != tune.cache_key(b, 4)
    assert tune.cache_key(a, 4) != tune.cache_key(a, 5)
    assert tune.cache_key(a, 4) != tune.cache_key(a, 4, ll.default_opts(chop_sections=4))
    assert tune.cache_key(a, 4, None, "x") != tune.cache_key(a, 4, None, "y")
    hash(tune.cache_key(a, 4))


def test_choice_prefers_fewer_fits_within_the_tie():
    W = lambda f, o=0: ll.Launch(32, f, o)  # noqa: E731
    blk = ll.Launch(512, 0, 0)
    # the fastest wins when nothing else is within 1 %
    assert tune.choose({W(6): 1.00, W(3): 1.05, blk: 2.0}) == W(6)
    # within the tie: the fewest fits per block, then work order 0
    assert tune.choose({W(6): 1.000, W(3): 1.005, W(2): 1.2}) == W(3)
    assert tune.choose({W(3, 1): 1.000, W(3, 0): 1.009}) == W(3, 0)
    # the one-warp shape before the block shape at equal time
    assert tune.choose({blk: 1.0, W(6): 1.0}) == W(6)
    assert tune.choose({blk: 1.0, W(6): 1.5}) == blk
    # smaller groups first within the tie, then fewer fits per block
    G2 = ll.Launch(64, 6, 0)
    G4 = ll.Launch(128, 4, 0)
    assert tune.choose({G4: 1.0, G2: 1.005, W(6): 1.5}) == G2
    assert tune.choose({G4: 1.0, G2: 1.2}) == G4
    assert tune.choose({G2: 1.0, W(6): 1.009}) == W(6)
    # a wider tie admits slower shapes
    assert tune.choose({W(6): 1.0, W(2): 1.04}, tie=0.05) == W(2)


def test_sample_subset_keeps_every_kth_problem():
    import numpy as np
    import torch
    from paper_2510_15649_gb300 import synth
    b = synth.batched_like(10, 5, 30, 2, 6, R=100, P=6, seed=2)
    pr = ll.Problems.from_numpy(b, device="cpu")
    lam = torch.arange(10 * 3, dtype=torch.float32).reshape(10, 3)
    sub, sl = tune._subset(pr, lam, 3)
    qs = [0, 3, 6, 9]
    off = b["offsets"]
    so = sub.offsets.numpy()
    assert sub.B == 4 and len(so) == 5
    for k, q in enumerate(qs):
        rows = b["row_idx"][off[q]:off[q + 1]]
        assert np.array_equal(sub.row_idx.numpy()[so[k]:so[k + 1]], rows)
        assert np.array_equal(sub.y.numpy()[so[k]:so[k + 1]], b["y"][off[q]:off[q + 1]])
        assert sub.p.numpy()[k] == b["p"][q]
        assert np.array_equal(sl[k].numpy(), lam[q].numpy())
    assert so[-1] == sub.y.numel()  # the library's rule: the set ends at its row count
    assert sub.X is pr.X and sub.n_max == pr.n_max

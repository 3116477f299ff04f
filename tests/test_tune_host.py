"""Host logic of the autotuner: candidate launch shapes (no GPU: the
library's launch_shape entry point touches no device)."""
from paper_2510_15649_gb300 import ladlasso as ll
from paper_2510_15649_gb300 import tune


class Pr:  # the fields candidates() reads
    def __init__(self, P, n_max):
        self.P, self.n_max = P, n_max


def test_candidates_cover_both_shapes_and_orders_when_both_fit():
    c = tune.candidates(Pr(32, 2000))
    warp = [x for x in c if x.group_threads == 32]
    block = [x for x in c if x.group_threads == 512]
    _, fmax, _ = ll.launch_shape(Pr(32, 2000))
    assert {x.fits_per_block for x in warp} == set(range(max(1, fmax // 3), fmax + 1))
    assert {x.work_order for x in warp} == {0, 1}
    assert block == [ll.Launch(512, 0, 0), ll.Launch(512, 0, 1)]
    assert len(set(c)) == len(c)


def test_long_problems_only_get_the_block_shape():
    c = tune.candidates(Pr(128, 20000))
    assert c and all(x.group_threads == 512 for x in c)


def test_no_candidate_beyond_every_shape():
    assert tune.candidates(Pr(128, 10 ** 6)) == []


def test_cache_round_trips_through_json(tmp_path):
    tune._cache.clear()
    key = ("GB300", 32, 2000, 4096, 16, False)
    times = {ll.Launch(32, 3, 0): 1.046, ll.Launch(32, 5, 1): 1.107, ll.Launch(512, 0, 0): 2.0}
    tune._cache[key] = (ll.Launch(32, 3, 0), times)
    path = str(tmp_path / "tune.json")
    tune.save_cache(path)
    tune._cache.clear()
    assert tune.load_cache(path) == 1
    choice, t2 = tune._cache[key]
    assert choice == ll.Launch(32, 3, 0) and t2 == times
    tune._cache.clear()

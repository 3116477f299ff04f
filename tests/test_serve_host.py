"""Host logic of the server: the problem set that computes lambda_max for
newly admitted slots must pass the library's offset rule (non-negative,
non-decreasing, last offset equal to the pool's row count) while each
problem still starts at its own slot and has room for a full slot."""
import numpy as np
import pytest

from paper_2510_15649_gb300.serve import admission_offsets


def _library_accepts(offsets, total_rows):
    # the rule ladlasso_lambda_max / ladlasso_fit_batched apply to offsets
    o = np.asarray(offsets, np.int64)
    return bool(np.all(o >= 0) and np.all(o <= total_rows) and np.all(np.diff(o) >= 0)
                and o[-1] == total_rows)


@pytest.mark.parametrize("slots", [[0], [0, 1, 2], [3], [1, 5, 6], [7], [0, 7], [2, 4, 6, 7]])
def test_admission_offsets_pass_the_library_rule(slots):
    S, cap = 8, 300
    off = admission_offsets(np.array(slots), cap, S)
    assert len(off) == len(slots) + 1
    assert _library_accepts(off, S * cap)
    assert np.array_equal(off[:-1], np.array(slots) * cap)
    assert np.all(np.diff(off) >= cap)


def test_offsets_ending_at_the_last_new_slot_were_rejected():
    # the form that ended the set at (last new slot + 1) * cap fails the
    # rule whenever the last slot of the pool is not among the new ones
    S, cap, ss = 8, 300, np.array([0, 2])
    assert not _library_accepts(np.append(ss * cap, (ss[-1] + 1) * cap), S * cap)


# ------------------------------------------------------------------ the
# request loop on CPU tensors, with the four library calls the server makes
# replaced by a fake that checks each call against the library's rules


class FakeLibrary:
    """Stands in for ladlasso.workspace / lambda_max / lambda_path / fit.
    lambda_max follows its definition (max_j |X_j^T sign(y)| over the rows
    a problem uses) so each result can be traced to its own request's data;
    `fit` moves b by +1 on the used columns per call, so the warm start a
    slot carries from step to step is visible in the results."""

    def __init__(self, fail_at_step=None):
        self.calls = 0
        self.fail_at_step = fail_at_step
        self.max_used = 0
        self.positions = []  # per launch: positions each active slot took

    def workspace(self, pr, L=1):
        import torch
        return torch.empty(16, dtype=torch.uint8)

    def lambda_max(self, pr, ws=None, stream=None):
        import torch
        off = pr.offsets.numpy()
        nr = pr.n_rows.numpy()
        p = pr.p.numpy()
        X, y = pr.X.numpy(), pr.y.numpy()
        B = len(off) - 1
        out = np.full(B, np.nan, np.float32)
        # the library's offset rule; a set that breaks it is bad input
        if _library_accepts(off, y.shape[0]) and np.all(nr <= np.diff(off)):
            for q in range(B):
                rows = slice(off[q], off[q] + nr[q])
                out[q] = np.abs(X[rows, :p[q]].T @ np.sign(y[rows])).max()
        return torch.from_numpy(out)

    def lambda_path(self, lmax, L, ratio=1e-3, stream=None):
        import torch
        t = np.arange(L) / max(1, L - 1)
        return torch.from_numpy((lmax.numpy()[:, None] * ratio ** t).astype(np.float32))

    def fit(self, pr, lambdas, *, b_init=None, opts=None, ws=None, out=None, launch=None, **kw):
        from paper_2510_15649_gb300 import ladlasso as ll
        self.calls += 1
        if self.calls == self.fail_at_step:
            raise ll.LadLassoError("injected failure")
        lam = lambdas.numpy()  # [S, K]: a slot's positions first, NaN after
        nr, p = pr.n_rows.numpy(), pr.p.numpy()
        ok = np.isfinite(lam)
        active = np.nonzero(ok[:, 0])[0]
        self.positions.append(ok.sum(axis=1)[active].tolist())
        # valid positions come first, then NaN
        assert np.all(ok[:, 1:] <= ok[:, :-1]), "a valid position after a NaN one"
        assert np.all(nr[active] > 0), "a slot with a lambda holds no rows"
        # the server's contract: idle slots are passed with NaN and 0 rows
        assert np.all(nr[~ok[:, 0]] == 0), "an idle slot still passes rows"
        self.max_used = max(self.max_used, int((nr[active] * p[active]).sum()))
        bcur = b_init.numpy().copy()  # [S, P]: each position warm-starts the next
        b, obj, st = out["b"].numpy(), out["obj"].numpy(), out["status"].numpy()
        for q in range(lam.shape[0]):
            for l in range(lam.shape[1]):
                b[q, l] = 0.0
                if ok[q, l]:
                    bcur[q, :p[q]] += 1.0
                    b[q, l, :p[q]] = bcur[q, :p[q]]
                    obj[q, l], st[q, l] = lam[q, l], 0
                else:
                    obj[q, l], st[q, l] = 0.0, 2
        return out


@pytest.fixture
def fake(monkeypatch):
    from paper_2510_15649_gb300 import ladlasso as ll

    def install(**kw):
        f = FakeLibrary(**kw)
        for name in ("workspace", "lambda_max", "lambda_path", "fit"):
            monkeypatch.setattr(ll, name, getattr(f, name))
        return f
    return install


def _trace(n=24, seed=3):
    from paper_2510_15649_gb300 import synth
    return synth.serve_trace(rate=4000.0, seconds=1.0, seed=seed, n_hi=300, p_hi=8,
                             max_requests=n)


def test_every_request_is_fitted_on_its_own_data_and_warm_started(fake):
    from paper_2510_15649_gb300.serve import Server
    f = fake()
    trace = _trace()
    L = 3
    srv = Server(slots=4, cap=300, P=8, L=L, device="cpu")
    results, st = srv.run(trace, time_scale=1.0)
    assert st.completed == len(trace) == len(results) and st.bad_fits == 0
    assert st.fits == len(trace) * L and st.max_active <= 4
    assert sorted(r.rid for r in results) == list(range(len(trace)))
    for r in results:
        X, y = trace[r.rid]["X"], trace[r.rid]["y"]
        # lambda_max of this request's own rows and columns, then its path
        lmax = np.abs(X.T @ np.sign(y)).max()
        np.testing.assert_allclose(r.lambdas[0], lmax, rtol=1e-5)
        np.testing.assert_allclose(r.lambdas, lmax * 1e-3 ** (np.arange(L) / (L - 1)), rtol=1e-5)
        # b starts from zero (slots are reused) and is carried step to step
        assert r.b.shape == (L, X.shape[1])
        for l in range(L):
            assert np.all(r.b[l] == l + 1.0)
        assert np.array_equal(r.obj, r.lambdas) and np.all(r.status == 0)
        assert r.t_done >= r.t_arrival
    assert f.calls == st.steps


def test_small_requests_take_several_positions_per_launch(fake):
    from paper_2510_15649_gb300.serve import Server
    f = fake()
    rng = np.random.default_rng(4)
    # one long request and short ones arriving together: the short ones
    # finish their 4-position paths in one launch, the long one takes one
    # position per launch; every warm start still carries through
    mk = lambda n, p: dict(t=0.0, X=rng.standard_normal((n, p)).astype(np.float32),  # noqa: E731
                           y=rng.standard_normal(n).astype(np.float32))
    trace = [mk(280, 8)] + [mk(20, 2) for _ in range(3)]
    srv = Server(slots=4, cap=300, P=8, L=4, device="cpu")
    results, st = srv.run(trace, time_scale=0.0)
    assert st.completed == 4 and st.fits == 16 and st.steps == 4
    assert f.positions[0] == [1, 4, 4, 4] or sorted(f.positions[0]) == [1, 4, 4, 4]
    assert all(x == [1] for x in f.positions[1:])
    for r in results:
        for l in range(4):
            assert np.all(r.b[l] == l + 1.0)
    # one position per launch when asked
    f2 = fake()
    srv = Server(slots=4, cap=300, P=8, L=4, device="cpu", positions_per_step=1)
    results, st = srv.run(trace, time_scale=0.0)
    assert st.steps == 4 and all(set(x) == {1} for x in f2.positions)
    assert all(np.all(r.b[l] == l + 1.0) for r in results for l in range(4))


def test_memory_budget_bounds_the_active_work(fake):
    from paper_2510_15649_gb300.serve import Server
    f = fake()
    trace = _trace(n=16, seed=5)
    budget = int(1.5 * max(r["X"].size for r in trace))
    srv = Server(slots=8, cap=300, P=8, L=2, budget_floats=budget, device="cpu")
    results, st = srv.run(trace, time_scale=0.0)  # every request arrives at once
    assert st.completed == len(trace) and st.bad_fits == 0
    assert f.max_used <= budget and st.queued_max >= 2
    assert srv.used == 0 and len(srv.free) == 8  # every slot and byte returned


def test_injected_library_failure_reaches_the_caller(fake):
    from paper_2510_15649_gb300 import ladlasso as ll
    from paper_2510_15649_gb300.serve import Server
    fake(fail_at_step=3)
    srv = Server(slots=4, cap=300, P=8, L=4, device="cpu")
    with pytest.raises(ll.LadLassoError, match="injected failure"):
        srv.run(_trace(n=8), time_scale=0.0)


def test_request_beyond_slot_capacity_is_refused_on_the_host(fake):
    from paper_2510_15649_gb300.serve import Server
    fake()
    rng = np.random.default_rng(1)
    big = dict(t=0.0, X=rng.standard_normal((301, 4)).astype(np.float32),
               y=rng.standard_normal(301).astype(np.float32))
    wide = dict(t=0.0, X=rng.standard_normal((20, 9)).astype(np.float32),
                y=rng.standard_normal(20).astype(np.float32))
    for req in (big, wide):
        with pytest.raises(ValueError):
            Server(slots=2, cap=300, P=8, L=2, device="cpu").run([req])


def test_request_beyond_the_memory_budget_is_refused_not_queued_forever(fake):
    from paper_2510_15649_gb300.serve import Server
    fake()
    rng = np.random.default_rng(2)
    req = dict(t=0.0, X=rng.standard_normal((100, 4)).astype(np.float32),
               y=rng.standard_normal(100).astype(np.float32))
    srv = Server(slots=2, cap=300, P=8, L=2, budget_floats=399, device="cpu")
    with pytest.raises(ValueError, match="memory budget"):
        srv.run([req])
    # exactly at the budget it is served
    results, st = Server(slots=2, cap=300, P=8, L=2, budget_floats=400, device="cpu").run([req])
    assert st.completed == 1


# ------------------------------------------------------------------ slot classes


def _record_admissions(pools, log):
    for pl in pools:
        orig = pl._admit

        def wrapped(reqs, rids, pl=pl, orig=orig):
            out = orig(reqs, rids)
            # the smallest class's free slots when this admission happens
            # (each round admits the classes smallest first)
            log.append((pl.cap, pl.P, list(rids), len(pools[0].free),
                        sum(q.used for q in pools)))
            return out
        pl._admit = wrapped


def test_slot_classes_serve_every_request_from_a_class_that_holds_it(fake):
    from paper_2510_15649_gb300.serve import ClassedServer
    fake()
    trace = _trace(n=40, seed=7)
    L = 3
    srv = ClassedServer([(2, 300, 8), (3, 100, 8)], L=L, device="cpu")
    assert [pl.cap for pl in srv.pools] == [100, 300]  # smallest class first
    log = []
    _record_admissions(srv.pools, log)
    results, st = srv.run(trace, time_scale=0.0)  # every request waiting at once
    assert st.completed == len(trace) and st.bad_fits == 0
    assert sorted(r.rid for r in results) == list(range(len(trace)))
    where = {}
    for cap, P, rids, _, _ in log:
        for rid in rids:
            n, p = trace[rid]["X"].shape
            assert n <= cap and p <= P
            where[rid] = cap
    small = [i for i, r in enumerate(trace) if r["X"].shape[0] <= 100]
    assert small and any(where[i] == 100 for i in small)
    # a short request in the large class only while the small class was full
    fallbacks = 0
    for cap, P, rids, small_free, _ in log:
        if cap == 300 and any(trace[rid]["X"].shape[0] <= 100 for rid in rids):
            assert small_free == 0
            fallbacks += 1
    assert fallbacks > 0  # with every request waiting, the small class overflows
    for r in results:  # own data, own path, warm starts, as with one pool
        X, y = trace[r.rid]["X"], trace[r.rid]["y"]
        lmax = np.abs(X.T @ np.sign(y)).max()
        np.testing.assert_allclose(r.lambdas[0], lmax, rtol=1e-5)
        for l in range(L):
            assert np.all(r.b[l] == l + 1.0)


def test_slot_classes_share_one_memory_budget(fake):
    from paper_2510_15649_gb300.serve import ClassedServer
    fake()
    trace = _trace(n=24, seed=8)
    budget = int(1.5 * max(r["X"].size for r in trace))
    srv = ClassedServer([(4, 300, 8), (4, 100, 8)], L=2, budget_floats=budget, device="cpu")
    log = []
    _record_admissions(srv.pools, log)
    results, st = srv.run(trace, time_scale=0.0)
    assert st.completed == len(trace)
    assert max(u for *_, u in log) <= budget
    assert all(pl.used == 0 for pl in srv.pools)


def test_slot_classes_refuse_a_request_no_class_holds(fake):
    from paper_2510_15649_gb300.serve import ClassedServer
    fake()
    rng = np.random.default_rng(3)
    big = dict(t=0.0, X=rng.standard_normal((301, 4)).astype(np.float32),
               y=rng.standard_normal(301).astype(np.float32))
    with pytest.raises(ValueError, match="slot capacity"):
        ClassedServer([(2, 100, 8), (2, 300, 8)], L=2, device="cpu").run([big])
    with pytest.raises(ValueError):
        ClassedServer([], device="cpu")


def test_broken_bookkeeping_raises_instead_of_waiting_forever(fake):
    # a server whose free-slot list was lost can admit nothing while nothing
    # runs: it must report that, not spin
    from paper_2510_15649_gb300.serve import Server
    fake()
    srv = Server(slots=2, cap=300, P=8, L=2, device="cpu")
    srv.free = []
    with pytest.raises(RuntimeError, match="stalled"):
        srv.run(_trace(n=2), time_scale=0.0)

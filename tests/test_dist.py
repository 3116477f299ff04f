"""Host logic of the N > 1 path on CPU: problems sharded by count or by
cost, batches cut into per-rank problem sets, and two gloo ranks that
cover a batch exactly once and agree on the job time (max over ranks)."""
import os
import socket

import numpy as np
import pytest

from paper_2510_15649_gb300 import synth
from paper_2510_15649_gb300.dist import (cost_shard_range, cost_share, covered_once, gather_lists,
                                         problem_cost,
                                         max_over_ranks, route_requests, shard_batch, shard_range,
                                         sum_over_ranks)


def test_shards_cover_every_problem_once():
    for B in [0, 1, 7, 4096, 4097]:
        for world in [1, 2, 3, 8]:
            seen = []
            for r in range(world):
                lo, hi = shard_range(B, r, world)
                assert hi - lo in (B // world, B // world + 1)
                seen.extend(range(lo, hi))
            assert seen == list(range(B))
    with pytest.raises(ValueError):
        shard_range(4, 2, 2)


def test_problem_cost_is_steps_times_rows_plus_fixed_part():
    b = dict(offsets=np.array([0, 10, 10, 2010]), p=np.array([3, 1, 32]))
    assert problem_cost(b, 1).tolist() == [3 * 1034.0, 1024.0, 32 * 3024.0]
    assert problem_cost(b, 16).tolist() == [16 * 3 * 1034.0, 16 * 1024.0, 16 * 32 * 3024.0]


def _ranges(cost, world):
    return [cost_shard_range(cost, r, world) for r in range(world)]


def test_cost_shards_cover_and_balance():
    b = synth.batched(B=512, seed=1)
    n = np.diff(b["offsets"])
    cost = n * b["p"] * 16.0  # n * p * L
    total, cmax = cost.sum(), cost.max()
    for world in range(1, 9):
        rs = _ranges(cost, world)
        assert rs[0][0] == 0 and rs[-1][1] == len(cost)
        assert all(rs[k][1] == rs[k + 1][0] for k in range(world - 1))  # contiguous
        shares = [cost[lo:hi].sum() for lo, hi in rs]
        assert max(abs(s - total / world) for s in shares) <= cmax
        # never worse than splitting by problem count
        eq = [cost[lo:hi].sum() for lo, hi in (shard_range(len(cost), r, world) for r in range(world))]
        assert max(shares) <= max(eq) + 1e-9 * total
    # one dominant problem gets a rank to itself
    c = np.array([1.0] * 8 + [100.0] + [1.0] * 8)
    assert (8, 9) in _ranges(c, 3) or (8, 9) in _ranges(c, 4)


def test_cost_shard_edge_cases():
    assert _ranges([], 3) == [(0, 0)] * 3
    assert _ranges([0.0, 0.0, 0.0], 2) == [shard_range(3, r, 2) for r in range(2)]
    one = _ranges([5.0], 4)  # more ranks than problems: one rank gets it, the rest none
    assert sorted(hi - lo for lo, hi in one) == [0, 0, 0, 1] and one[0][0] == 0 and one[-1][1] == 1
    with pytest.raises(ValueError):
        cost_shard_range([1.0, -1.0], 0, 2)
    with pytest.raises(ValueError):
        cost_shard_range([1.0], 2, 2)


def test_shard_batch_reassembles_the_batch():
    b = synth.batched_like(9, 5, 40, 2, 6, R=60, P=6, seed=3)
    cuts = [(0, 4), (4, 4), (4, 9)]
    parts = [shard_batch(b, lo, hi) for lo, hi in cuts]
    assert np.array_equal(np.concatenate([p["y"] for p in parts]), b["y"])
    assert np.array_equal(np.concatenate([p["row_idx"] for p in parts]), b["row_idx"])
    assert np.array_equal(np.concatenate([p["p"] for p in parts]), b["p"])
    for (lo, hi), p in zip(cuts, parts):
        assert p["offsets"][0] == 0 and len(p["offsets"]) == hi - lo + 1
        assert np.array_equal(np.diff(p["offsets"]), np.diff(b["offsets"])[lo:hi])
        assert p["X"] is b["X"]
    # contiguous problems (slots are rows of X): X is sliced with y
    L = synth.large(B=3, n=50, p=12)
    mid = shard_batch(L, 1, 2)
    assert np.array_equal(mid["X"], L["X"][50:100]) and mid["row_idx"] is None
    assert np.array_equal(mid["offsets"], [0, 50])


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = shard_range(10, rank, world)
    t = max_over_ranks(1.0 + rank, dist)
    total = sum_over_ranks(1.0 + rank, dist)
    # cost-balanced shares of one batch: every problem fitted exactly once
    import torch
    b = synth.batched_like(40, 5, 200, 2, 8, R=250, P=8, seed=7)
    cost = problem_cost(b, 1)
    clo, chi = cost_shard_range(cost, rank, world)
    part = shard_batch(b, clo, chi)
    done = torch.zeros(40, dtype=torch.int64)
    done[clo:chi] = 1
    dist.all_reduce(done)
    mine = float(problem_cost(part, 1).sum())
    # the benchmark's strong-scaling share: the same cut with L = 16, and
    # the coverage check over both ranks (a planted overlap fails it)
    sb, (slo, shi) = cost_share(b, 16, rank, world)
    assert (slo, shi) == (clo, chi) and np.array_equal(sb["y"], part["y"])
    ok = covered_once(slo, shi, 40, dist)
    overlap = covered_once(0, shi if rank == 0 else 40, 40, dist)
    out.put((rank, lo, hi, t, done.tolist(), mine, float(cost.sum()), total, ok, overlap))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time():
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[3] for r in res] == [2.0, 2.0]
    assert (res[0][1], res[0][2], res[1][1], res[1][2]) == (0, 5, 5, 10)
    assert res[0][4] == [1] * 40 and res[1][4] == [1] * 40
    assert res[0][5] + res[1][5] == res[0][6]
    assert [r[7] for r in res] == [3.0, 3.0]
    assert [r[8] for r in res] == [True, True] and [r[9] for r in res] == [False, False]
    assert covered_once(0, 5, 5) and not covered_once(0, 4, 5)  # no process group
    assert sum_over_ranks(2.5) == 2.5 and max_over_ranks(2.5) == 2.5  # no process group


def test_route_requests_balances_load_in_arrival_order():
    assert route_requests([], 3).tolist() == []
    assert route_requests([5.0, 1.0, 1.0, 1.0], 2).tolist() == [0, 1, 1, 1]
    assert route_requests([1.0] * 6, 3).tolist() == [0, 1, 2, 0, 1, 2]
    rng = np.random.default_rng(0)
    w = rng.uniform(1.0, 100.0, 500)
    for world in (1, 2, 4, 8):
        r = route_requests(w, world)
        assert set(r.tolist()) <= set(range(world))
        loads = np.bincount(r, weights=w, minlength=world)
        # greedy least-loaded: every rank within one request of the others
        assert loads.max() - loads.min() <= w.max()
    with pytest.raises(ValueError):
        route_requests([1.0, -1.0], 2)
    with pytest.raises(ValueError):
        route_requests([1.0], 0)
    assert gather_lists([1, 2]) == [1, 2]  # no process group


def _serve_worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2510_15649_gb300 import ladlasso as ll
    from paper_2510_15649_gb300.serve import Server, serve_distributed
    from test_serve_host import FakeLibrary
    f = FakeLibrary()
    for name in ("workspace", "lambda_max", "lambda_path", "fit"):
        setattr(ll, name, getattr(f, name))
    trace = synth.serve_trace(rate=4000.0, seconds=1.0, seed=9, n_hi=300, p_hi=8,
                              max_requests=30)
    srv = Server(slots=4, cap=300, P=8, L=3, device="cpu")
    results, st = serve_distributed(srv, trace, rank, world, dist, time_scale=0.0)
    lam_ok = all(np.isclose(r.lambdas[0], np.abs(trace[r.rid]["X"].T @ np.sign(trace[r.rid]["y"])).max(),
                            rtol=1e-5) for r in results)
    out.put((rank, sorted(r.rid for r in results), st.completed, st.fits, len(st.latencies),
             st.wall, lam_ok))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_serve_one_trace_between_them():
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_serve_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    trace = synth.serve_trace(rate=4000.0, seconds=1.0, seed=9, n_hi=300, p_hi=8, max_requests=30)
    route = route_requests([r["X"].size for r in trace], 2)
    # each request served once, by the rank it was routed to, on its own data
    for rank, rids, *_ in res:
        assert rids == [i for i in range(30) if route[i] == rank]
        assert rids
    assert sorted(res[0][1] + res[1][1]) == list(range(30))
    assert all(r[6] for r in res)
    # the merged report is the same on both ranks: every request, every fit
    for r in res:
        assert r[2] == 30 and r[3] == 30 * 3 and r[4] == 30
    assert res[0][5] == res[1][5]

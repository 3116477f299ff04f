"""Host logic of the N > 1 path on CPU: problems sharded by count or by
cost, batches cut into per-rank problem sets, and two gloo ranks that
cover a batch exactly once and agree on the job time (max over ranks)."""
import os
import socket

import numpy as np
import pytest

from paper_2510_15649_gb300 import synth
from paper_2510_15649_gb300.dist import (cost_shard_range, max_over_ranks, shard_batch, shard_range,
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
    cost = np.diff(b["offsets"]) * b["p"]
    clo, chi = cost_shard_range(cost, rank, world)
    part = shard_batch(b, clo, chi)
    done = torch.zeros(40, dtype=torch.int64)
    done[clo:chi] = 1
    dist.all_reduce(done)
    mine = float(np.sum(np.diff(part["offsets"]) * part["p"]))
    out.put((rank, lo, hi, t, done.tolist(), mine, float(cost.sum()), total))
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
    assert sum_over_ranks(2.5) == 2.5 and max_over_ranks(2.5) == 2.5  # no process group

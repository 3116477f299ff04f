"""Host logic of the N > 1 path on CPU: two gloo ranks shard a batch and
agree on the job time (max over ranks)."""
import os
import socket

import numpy as np
import pytest

from paper_2510_15649_gb300.dist import max_over_ranks, shard_range


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


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = shard_range(10, rank, world)
    t = max_over_ranks(1.0 + rank, dist)
    out.put((rank, lo, hi, t))
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

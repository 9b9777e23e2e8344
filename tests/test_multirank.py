"""The multi-rank path of the sweep (sharding and reporting) with world_size 2 on the gloo
backend (CPU): no GPU involved."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2307_05590_gb300 import shard
    from workloads import reduced_dictionary
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rs = np.array([o.r for o in reduced_dictionary(60, seed=20230711)])
        costs = shard.sweep_cost(rs, 2000)
        mine = shard.balanced_split(costs, world)[rank]
        # every rank sees the same split; its load and the totals agree across ranks
        load = float(costs[mine].sum())
        total = shard.sum_over_ranks(load)
        worst = shard.max_over_ranks(load)
        count = shard.sum_over_ranks(len(mine))
        step = shard.max_over_ranks(0.1 * (rank + 1))  # the slowest rank's step time
        out[rank] = (load, total, worst, count, step, mine)
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_and_reporting():
    import torch.multiprocessing as mp
    from paper_2307_05590_gb300 import shard
    from workloads import reduced_dictionary
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    rs = np.array([o.r for o in reduced_dictionary(60, seed=20230711)])
    costs = shard.sweep_cost(rs, 2000)
    assert sorted(out[0][5] + out[1][5]) == list(range(60))       # every object exactly once
    for rank in range(world):
        load, total, worst, count, step, _ = out[rank]
        assert np.isclose(total, costs.sum()) and count == 60
        assert np.isclose(worst, max(out[0][0], out[1][0]))
        assert step == pytest.approx(0.2)                            # max over ranks
    assert max(out[0][0], out[1][0]) <= 1.01 * costs.sum() / world   # balanced within 1 %


def test_balanced_split_edge_cases():
    from paper_2307_05590_gb300 import shard
    assert shard.balanced_split([], 3) == [[], [], []]
    assert shard.balanced_split([5.0], 2) in ([[0], []], [[], [0]])
    parts = shard.balanced_split(np.ones(10), 4)
    assert sorted(len(p) for p in parts) == [2, 2, 3, 3]
    with pytest.raises(ValueError):
        shard.balanced_split([1.0], 0)
    assert shard.max_over_ranks(1.5) == 1.5 and shard.sum_over_ranks(2.0) == 2.0  # no process group

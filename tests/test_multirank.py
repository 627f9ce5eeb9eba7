"""The N > 1 host logic (replicas, no data exchange) on world-size-2 gloo ranks (CPU)."""
import os
import socket

import pytest

from paper_2103_02309_gb300.shard import lpt_assign, max_over_ranks

torch = pytest.importorskip("torch")


def test_lpt_assign_bound_and_cover():
    import random
    rnd = random.Random(5)
    for world in (1, 2, 3, 8):
        costs = [rnd.lognormvariate(0, 2) for _ in range(32)]
        rank = lpt_assign(costs, world)
        assert len(rank) == len(costs) and set(rank) <= set(range(world))
        load = [sum(c for c, r in zip(costs, rank) if r == k) for k in range(world)]
        lower = max(max(costs), sum(costs) / world)      # no schedule does better
        assert max(load) <= 4 / 3 * lower + 1e-9
    assert lpt_assign([3, 3, 2, 2, 2], 2) == [0, 1, 0, 1, 0]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, costs, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [i for i, r in enumerate(lpt_assign(costs, world)) if r == rank]
        got = [None] * world
        dist.all_gather_object(got, mine)
        step_ms = 10.0 + 5.0 * rank                          # a stand-in for each rank's time
        out[rank] = (got, max_over_ranks(step_ms))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_meshes_and_max_time():
    import torch.multiprocessing as mp
    costs = [5.0, 1.0, 7.0, 2.0, 2.0, 9.0, 0.5]
    world = 2
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), costs, out), nprocs=world,
                           start_method="spawn")
        res = dict(out)
    for rank in range(world):
        shards, tmax = res[rank]
        assert sorted(i for s in shards for i in s) == list(range(len(costs)))
        assert tmax == 15.0
    assert res[0][0] == res[1][0]

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


def test_tile_ranges_cover_each_ray_once():
    from paper_2103_02309_gb300.shard import tile_range
    for n in (0, 1, 31, 32, 33, 4096, 1920 * 1080, 2048 * 2048 + 5):
        for world in (1, 2, 3, 4, 8):
            r = [tile_range(n, world, k) for k in range(world)]
            assert r[0][0] == 0 and r[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))        # contiguous, rank order
            assert all(lo % 32 == 0 and lo <= hi for lo, hi in r)      # whole warp tiles
            sizes = [hi - lo for lo, hi in r]
            assert max(sizes) - min(sizes) <= 32 + (32 - n % 32) % 32  # even up to one tile
    with pytest.raises(ValueError):
        tile_range(10, 2, 2)


def test_shard_seed_reproduces_the_frames_draws():
    """A rank's local counters with the shifted seed draw the same numbers
    as the whole frame's counters (SplitMix64 as a counter-based generator)."""
    import numpy as np
    from oracle.secondary import uniform
    from paper_2103_02309_gb300.shard import shard_seed
    seed = 0x5EED
    for first, per_hit in ((0, 1), (1024, 1), (777, 8), (2 ** 21, 8)):
        local = np.arange(0, 2 * 50 * per_hit, dtype=np.uint64)
        whole = local + np.uint64(2 * first * per_hit)
        assert np.array_equal(uniform(shard_seed(seed, first, per_hit), local), uniform(seed, whole))


def _frame_rank_main(rank, world, port, out):
    """One rank of a frame split by pixel tiles: its camera rays and their
    bounce rays, traced by the oracle (standing in for the device walk on
    this CPU-only machine), gathered to rank 0 in pixel order."""
    import numpy as np
    import torch.distributed as dist

    import oracle
    import scenegen as sg
    from oracle.secondary import hit_side, secondary_rays
    from paper_2103_02309_gb300.shard import gather_rows, shard_seed, tile_range
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = sg.make_config("tiny")
        om = oracle.OracleMesh(s.points, s.tets, s.tris)
        cam, _ = om.locate(np.array([s.camera.eye], np.float32), nthreads=1)
        o, d = sg.camera_rays(s.camera)
        lo, hi = tile_range(len(o), world, rank)
        w = om.trace(o[lo:hi], d[lo:hi], np.inf, cam[0], nthreads=1)
        side = hit_side(om.arrays()[2], w["tri"], w["tet"])
        # local counters, as a rank's device generator sees its own hit buffer
        o2, d2, t2, e2, _ = secondary_rays(s.points, s.tris, w["tri"], w["b1"], w["b2"], side,
                                           shard_seed(9, lo, 1), 1, np.inf)
        w2 = om.trace(o2, d2, t2, -1, e2, nthreads=1)
        prim = torch.from_numpy(np.stack([w["tri"], w["t"].view(np.int64).astype(np.int64)], 1))
        sec = torch.from_numpy(np.stack([w2["tri"], w2["t"].view(np.int64).astype(np.int64)], 1))
        g1, g2 = gather_rows(prim, world, rank), gather_rows(sec, world, rank)
        if rank == 0:
            out[0] = (g1.numpy(), g2.numpy())
        out[f"range{rank}"] = (lo, hi)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_one_frame_by_tiles_and_gather_hits():
    import numpy as np
    import torch.multiprocessing as mp

    import oracle
    import scenegen as sg
    from oracle.secondary import hit_side, secondary_rays
    world = 2
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_frame_rank_main, args=(world, _free_port(), out), nprocs=world,
                           start_method="spawn")
        res = dict(out)
    s = sg.make_config("tiny")
    n = s.camera.width * s.camera.height
    assert res["range0"] == (0, n // 2) and res["range1"] == (n // 2, n)
    # the whole frame in one process
    om = oracle.OracleMesh(s.points, s.tets, s.tris)
    cam, _ = om.locate(np.array([s.camera.eye], np.float32))
    o, d = sg.camera_rays(s.camera)
    w = om.trace(o, d, np.inf, cam[0])
    side = hit_side(om.arrays()[2], w["tri"], w["tet"])
    o2, d2, t2, e2, _ = secondary_rays(s.points, s.tris, w["tri"], w["b1"], w["b2"], side, 9, 1,
                                       np.inf)
    w2 = om.trace(o2, d2, t2, -1, e2)
    g1, g2 = res[0]
    assert np.array_equal(g1[:, 0], w["tri"]) and np.array_equal(g1[:, 1].view(np.float64), w["t"])
    assert np.array_equal(g2[:, 0], w2["tri"]) and np.array_equal(g2[:, 1].view(np.float64), w2["t"])

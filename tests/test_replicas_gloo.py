"""The N > 1 host path of bench.py on CPU: two gloo ranks, each with its own
seeded batch, the job time the slowest rank's, the value every rank's
targets over that time."""
import os

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import scenegen as G
        sc = G.c1_scene(0)
        t = bench.rank_targets(sc, 8, rank)
        ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        job_ms = bench.max_over_ranks(ms, dist, torch.device("cpu"))
        # every rank's batch, gathered only to check it here
        got = [torch.zeros(8 * 3, dtype=torch.int32) for _ in range(world)]
        dist.all_gather(got, torch.from_numpy(np.ascontiguousarray(t, dtype=np.int32).reshape(-1)))
        out[rank] = (job_ms, bench.job_value(8, world, job_ms),
                     [g.numpy().reshape(-1, 3).tolist() for g in got])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_nothing_and_time_the_slowest():
    world = 2
    port = 29500 + (os.getpid() % 2000)
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    import bench
    import scenegen as G
    sc = G.c1_scene(0)
    for r in range(world):
        job_ms, value, batches = res[r]
        assert job_ms == 15.0                      # the slowest rank's time, on every rank
        assert value == bench.job_value(8, world, 15.0) == 16 / 0.015
        for q in range(world):                     # each rank's batch is its own seeded draw
            assert batches[q] == bench.rank_targets(sc, 8, q).tolist()
    assert res[0][2][0] != res[0][2][1]            # the two ranks solve different targets


def test_one_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, None, torch.device("cpu")) == 12.5
    assert bench.job_value(64, 1, 100.0) == 640.0

"""The multi-rank path of bench.py on the CPU: two gloo ranks (replicas) reduce
their timings to the slowest rank, and each rank draws its own frames."""

import os

import numpy as np
import torch.multiprocessing as mp


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2009_00946_b300 import configs
    vals = [10.0 + rank, 5.0 * (1 - rank), 7.0, 1.0 + 2 * rank]
    got = bench.max_over_ranks(vals, dist, torch.device("cpu"))
    cfg = configs.c5_autograd()
    pool = bench.slope_pool(cfg, 1, seed=cfg["seed"] + 100 * rank)
    out.put((rank, got, float(pool.sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert res[0][1] == res[1][1] == [11.0, 5.0, 7.0, 3.0]
    assert res[0][2] != res[1][2]          # each replica gets its own frames


def test_max_over_ranks_without_process_group():
    import bench
    assert bench.max_over_ranks(np.array([1.5, 2.0]), None, None) == [1.5, 2.0]

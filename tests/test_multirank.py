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


class _StubBatch:
    """CPU stand-in for fewha.Batch in the sharding test: the 'layers' of
    instance i are i + k / size (k = 0..size-1), so a gathered array shows
    which instance it came from and where it was cut."""

    def __init__(self, cfgs):
        self.cfgs = cfgs

    def layers(self):
        out = []
        for c in self.cfgs:
            i = int(c["name"].rsplit("_", 1)[1])
            n = sum(l["n"] ** 2 for l in c["layers"])
            out.append(i + np.arange(n, dtype=np.float64) / n)
        return np.concatenate(out).astype(np.float32)

    def close(self):
        pass


def _shard_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2009_00946_b300 import configs, shard
    cfgs = configs.c4_batch(64)
    sb = shard.ShardedBatch(cfgs, rank, world, batch_factory=_StubBatch)
    local = torch.from_numpy(sb.batch.layers()) if sb.batch else torch.zeros(0)
    got = sb.gather_layers(local, dist, dst=0, device=torch.device("cpu"))
    out.put((rank, sb.mine, None if got is None else [float(a[0]) for a in got],
             None if got is None else [int(a.size) for a in got],
             None if got is None else [float(a[-1]) for a in got]))
    dist.barrier()
    dist.destroy_process_group()


def test_batch_instances_shard_across_two_gloo_ranks():
    """Instances partitioned over two ranks (no collective in the solve): a
    disjoint cover of all 64, balanced in cost, and the gathered layers land
    at the right instance with the right length on rank 0."""
    from paper_2009_00946_b300 import configs, shard
    cfgs = configs.c4_batch(64)
    costs = [shard.instance_cost(c) for c in cfgs]
    parts = shard.partition(costs, 2)
    assert sorted(parts[0] + parts[1]) == list(range(64))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(costs)          # LPT balance bound
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29600 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_shard_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=180) for _ in range(2)], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] == parts[0] and res[1][1] == parts[1]   # every rank computes the same partition
    firsts, sizes, lasts = res[0][2], res[0][3], res[0][4]
    assert res[1][2] is None                                 # only rank 0 receives
    want_sizes = shard.layer_sizes(cfgs)
    for i in range(64):
        assert sizes[i] == want_sizes[i]
        assert firsts[i] == float(np.float32(i))
        assert abs(lasts[i] - (i + (want_sizes[i] - 1) / want_sizes[i])) < 1e-3


def test_partition_single_rank_and_more_ranks_than_instances():
    from paper_2009_00946_b300 import shard
    assert shard.partition([5, 3, 9], 1) == [[0, 1, 2]]
    p = shard.partition([5, 3, 9], 5)
    assert sorted(sum(p, [])) == [0, 1, 2] and sum(1 for x in p if not x) == 2

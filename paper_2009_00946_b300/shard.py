"""Batched instances sharded across ranks (one process per GPU).

Independent tomography instances share nothing but the launch, so a batch
splits across GPUs with no collective in the solve: every rank builds one
fewha_batch over its own instances and advances it frame by frame; only the
results travel, gathered to one rank when wanted.  This module is host logic
only (the partition, the offsets, the gather); every step of the
reconstruction runs in the library's kernels.

Partition: longest-processing-time-first over a per-instance cost (the FP32
elements one frame reads and writes: n_iter (16 N + 4 NW) + S + 2 NW + 10 N,
N coefficients, NW sensor nodes, S slopes), each instance to the rank with the
smallest load so far; ties go to the lower rank, so every rank computes the
same partition from the configurations alone.
"""

from __future__ import annotations

import numpy as np


def instance_cost(cfg: dict, n_iter: int = 4) -> int:
    """FP32 elements one frame of Alg. 1 with n_iter PCG iterations moves."""
    N = sum(int(l["n"]) ** 2 for l in cfg["layers"])
    NW = sum((int(w["n_sub"]) + 1) ** 2 for w in cfg["wfs"])
    S = sum(2 * int(w["n_sub"]) ** 2 for w in cfg["wfs"])
    return int(n_iter * (16 * N + 4 * NW) + S + 2 * NW + 10 * N)


def partition(costs, world: int) -> list[list[int]]:
    """Instances per rank (ascending instance order within a rank)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = [int(c) for c in costs]
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def layer_sizes(cfgs) -> list[int]:
    return [sum(int(l["n"]) ** 2 for l in c["layers"]) for c in cfgs]


class ShardedBatch:
    """The share of a batch of instances that belongs to this rank.

    cfgs: every instance of the whole batch (each rank passes the same list);
    rank / world: this process's place.  `mine` lists this rank's instances;
    frame() takes their slopes (a list in the order of `mine`) and advances
    them by the batch's fused launches; gather_layers() returns, on rank dst, every
    instance's layers in global instance order."""

    def __init__(self, cfgs: list, rank: int, world: int, n_iter: int = 4, batch_factory=None, **batch_kw):
        self.cfgs = cfgs
        self.rank, self.world = int(rank), int(world)
        self.parts = partition([instance_cost(c, n_iter) for c in cfgs], self.world)
        self.mine = self.parts[self.rank]
        self.sizes = layer_sizes(cfgs)
        if batch_factory is None:
            from . import fewha
            batch_factory = fewha.Batch
        self.batch = batch_factory([cfgs[i] for i in self.mine], **batch_kw) if self.mine else None

    def close(self):
        if self.batch is not None:
            self.batch.close()
            self.batch = None

    def gather_layers(self, local_layers, dist, dst: int = 0, device=None):
        """local_layers: this rank's instances' layers concatenated (in the
        order of `mine`; a torch tensor on `device`, the process group's
        device).  Returns, on rank dst, a list of numpy arrays (one per
        instance, global order); None on the other ranks.  One all_gather of
        equal-length (padded) tensors."""
        import torch
        longest = max(sum(self.sizes[i] for i in p) for p in self.parts)
        buf = torch.zeros(max(longest, 1), dtype=torch.float32, device=device)
        n_mine = sum(self.sizes[i] for i in self.mine)
        if n_mine:
            buf[:n_mine] = local_layers.reshape(-1)[:n_mine].to(buf.device, torch.float32)
        got = [torch.empty_like(buf) for _ in range(self.world)]
        dist.all_gather(got, buf)
        if self.rank != dst:
            return None
        out: list = [None] * len(self.cfgs)
        for r, p in enumerate(self.parts):
            v = got[r].cpu().numpy()
            o = 0
            for i in p:
                out[i] = v[o:o + self.sizes[i]].copy()
                o += self.sizes[i]
        return out

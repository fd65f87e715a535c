"""Multi-GPU execution of the fill: one process per GPU, elements sharded across ranks.

Each element matrix of Eq. (2)/(4) of arXiv:1703.09619 depends only on that element's
geometry, material, orders and quadrature, so elements are independent units and the
ranks exchange no data on the fill's path: every rank fills its own elements into its
own output.  The collectives here are host-side bookkeeping only: a barrier around timed
regions and the maximum of the elapsed times over ranks.  Rank, world size and local GPU
come from the launcher's environment (RANK, WORLD_SIZE, LOCAL_RANK).

Two ways to use several GPUs:
* weak scaling (fixed work per GPU): every rank fills a batch of its own
  (``workloads.make(name, shard=rank)``);
* strong scaling (one batch split over GPUs): ``balanced_ranges`` cuts the batch into
  contiguous element ranges of nearly equal entry counts (orders may be uneven), and each
  rank fills ``wl.subset(range(lo, hi))``.
"""
from __future__ import annotations

import os

import numpy as np


def env():
    """(world, rank, local_rank) from the launcher's environment (1, 0, 0 without one)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str):
    """Join the process group (``nccl`` for GPU ranks, ``gloo`` for CPU) when world > 1."""
    world, rank, local = env()
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)
    return world, rank, local


def balanced_ranges(weights, world: int):
    """Contiguous [lo, hi) unit ranges, one per rank, covering all units in order, with
    the sum of ``weights`` per range as even as contiguity allows: cut r sits at the unit
    boundary closest to r/world of the total weight, so no range exceeds its share by
    more than the heaviest unit."""
    if world < 1:
        raise ValueError("world must be >= 1")
    w = np.asarray(weights, dtype=np.float64).reshape(-1)
    if (w < 0).any():
        raise ValueError("weights must be >= 0")
    n = w.size
    c = np.concatenate([[0.0], np.cumsum(w)])
    total = c[-1]
    cuts = [0]
    for r in range(1, world):
        target = total * r / world
        i = int(np.searchsorted(c, target, side="left"))
        i = min(max(i, 0), n)
        if i > 0 and abs(c[i - 1] - target) <= abs(c[i] - target):
            i -= 1
        cuts.append(max(i, cuts[-1]))
    cuts.append(n)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The maximum of ``x`` over all ranks (the whole job's time is its slowest rank's)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int, device=None) -> float:
    """The sum of ``x`` over all ranks (units processed by the whole job)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())

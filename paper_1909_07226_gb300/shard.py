"""Gridding and degridding of one plan partitioned over several processes.

Subgrids are independent of one another; only their sum into the master grid
couples them (Sect. 3.2 of the paper: every subgrid is gridded, transformed and
added on its own).  So one plan shards by subgrid:

* rank r of W takes a contiguous range of the plan's subgrids (plan order),
  cut where the running visibility-pixel count sum K_p L^2 crosses r/W of the
  total, so every rank gets about the same gridder work;
* gridding: each rank grids its range into a private grid (idg_grid_range),
  then one sum-reduce over the ranks gives the master grid on every rank;
* degridding: each rank degrids its range (idg_degrid_range) into a zeroed
  visibility buffer; the ranges' visibilities are disjoint, so the same sum
  assembles the full set on every rank.

The collective is torch.distributed's all_reduce of the buffers viewed as real
numbers (NCCL between GPUs, gloo on the CPU).  It is the only exchange step of
the path.  The range computation is host arithmetic; the per-range work is
whatever `run_range(first, count, out)` does (the library's range calls on a
GPU; tests substitute the FP64 oracle).
"""
from __future__ import annotations

from typing import Callable, List, Tuple

import numpy as np


def shard_ranges(kp, world: int) -> List[Tuple[int, int]]:
    """Contiguous (first, count) ranges of the plan's subgrids, one per rank.

    kp: K_p of every subgrid in plan order.  Range r ends at the first subgrid
    whose running K_p sum reaches (r + 1) / world of the total (integer
    arithmetic, so every process computes the same cut)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    kp = np.asarray(kp, dtype=np.int64)
    n = kp.shape[0]
    prefix = np.concatenate([[0], np.cumsum(kp)])
    total = int(prefix[-1])
    cuts = [0]
    for r in range(1, world):
        # smallest i with prefix[i] * world >= r * total
        i = int(np.searchsorted(prefix * world, r * total, side="left"))
        cuts.append(min(max(i, cuts[-1]), n))
    cuts.append(n)
    return [(cuts[r], cuts[r + 1] - cuts[r]) for r in range(world)]


def _all_reduce_sum(t, group=None):
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return t
    dist.all_reduce(torch.view_as_real(t) if t.is_complex() else t, op=dist.ReduceOp.SUM, group=group)
    return t


def sharded(kp, run_range: Callable[[int, int, object], None], out, group=None):
    """Run this rank's range into `out` (zeroed first), then sum `out` over the
    ranks of `group` (the default group if None; a single process runs the
    whole plan).  Returns `out`."""
    import torch.distributed as dist
    if dist.is_initialized():
        rank, world = dist.get_rank(group), dist.get_world_size(group)
    else:
        rank, world = 0, 1
    first, count = shard_ranges(kp, world)[rank]
    out.zero_()
    if count:
        run_range(first, count, out)
    return _all_reduce_sum(out, group)


def grid(plan, vis, flags, aterms, taper, grid_out, group=None, stream=None):
    """The master grid of the plan's visibilities on every rank (overwrites grid_out)."""
    from . import idg
    kp = plan.export()[:, idg.DESC_FIELDS - 1]
    return sharded(kp, lambda f, c, out: idg.grid_range(plan, f, c, vis, flags, aterms, taper, out, stream),
                   grid_out, group)


def degrid(plan, grid_in, flags, aterms, taper, vis_out, group=None, stream=None):
    """All the plan's model visibilities on every rank (overwrites vis_out; flagged
    and dropped visibilities 0, as idg_degrid)."""
    from . import idg
    kp = plan.export()[:, idg.DESC_FIELDS - 1]
    return sharded(kp, lambda f, c, out: idg.degrid_range(plan, f, c, grid_in, flags, aterms, taper, out, stream),
                   vis_out, group)

"""Partition of one plan over ranks (two gloo ranks on the CPU).

Each rank runs the FP64 oracle on its own contiguous range of subgrids and the
ranks sum their buffers with one all_reduce, exactly as the GPU path sums the
ranges that idg_grid_range / idg_degrid_range produce.  The partition plus the
sum must reproduce the single-process oracle grid and visibilities (to FP64
rounding: only the order of the additions differs).  The ranges themselves are
checked on the host: they tile the plan and split its work evenly.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload():
    from paper_1909_07226_gb300 import synthetic as syn
    return syn.make_small(seed=44, n_st=6, n_t=40, n_chan=5, L=16, N=128, max_t=12, n_slots=2, flag_p=0.1,
                          w_step=30.0, diameter_m=6000.0)


def _rank_main(rank, world, port, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      OMP_NUM_THREADS="2")
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from oracle import oracle as O
    from paper_1909_07226_gb300 import shard
    from paper_1909_07226_gb300 import synthetic as syn
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = _workload()
        op = O.plan(wl)
        kp = op.desc[:, O.D_KP]
        G = syn.random_grid(np.random.default_rng(5), op.n_w, wl.grid_size)

        def grid_range(f, c, out):
            out += torch.from_numpy(O.grid(wl, op, ids=np.arange(f, f + c)))

        def degrid_range(f, c, out):
            out += torch.from_numpy(O.degrid(wl, op, G, ids=np.arange(f, f + c)))

        g = torch.zeros((op.n_w, wl.grid_size, wl.grid_size, 4), dtype=torch.complex128)
        shard.sharded(kp, grid_range, g)
        v = torch.zeros(wl.vis.shape, dtype=torch.complex128)
        shard.sharded(kp, degrid_range, v)
        first, count = shard.shard_ranges(kp, world)[rank]
        out_q.put((rank, first, count, g.numpy(), v.numpy()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_reproduce_the_single_process_oracle():
    import torch.multiprocessing as mp
    from oracle import oracle as O
    O.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(2)), key=lambda t: t[0])
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    wl = _workload()
    op = O.plan(wl)
    G = __import__("paper_1909_07226_gb300.synthetic", fromlist=["x"]).random_grid(
        np.random.default_rng(5), op.n_w, wl.grid_size)
    ref_g = O.grid(wl, op)
    ref_v = O.degrid(wl, op, G)
    (_, f0, c0, g0, v0), (_, f1, c1, g1, v1) = res
    assert f0 == 0 and f0 + c0 == f1 and f1 + c1 == op.n_sub and c0 > 0 and c1 > 0
    assert op.n_w > 1
    for g, v in ((g0, v0), (g1, v1)):        # every rank holds the whole result
        assert np.max(np.abs(g - ref_g)) <= 1e-12 * np.max(np.abs(ref_g))
        assert np.max(np.abs(v - ref_v)) <= 1e-12 * np.max(np.abs(ref_v))
    # one rank's share alone is not the whole grid
    part = O.grid(wl, op, ids=np.arange(f0, f0 + c0))
    assert np.linalg.norm(part - ref_g) > 0.1 * np.linalg.norm(ref_g)


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_ranges_tile_the_plan_and_balance_the_work(world):
    from paper_1909_07226_gb300 import shard
    rng = np.random.default_rng(world)
    kp = rng.integers(1, 2048, size=997)
    r = shard.shard_ranges(kp, world)
    assert len(r) == world
    assert r[0][0] == 0 and sum(c for _, c in r) == len(kp)
    for (f, c), (f2, _) in zip(r, r[1:]):
        assert f + c == f2
    work = [int(kp[f:f + c].sum()) for f, c in r]
    # each cut lands within one subgrid of the ideal share
    assert max(work) - min(work) <= 2 * int(kp.max())
    assert sum(work) == int(kp.sum())


def test_ranges_degenerate_cases():
    from paper_1909_07226_gb300 import shard
    assert shard.shard_ranges([], 3) == [(0, 0), (0, 0), (0, 0)]
    assert shard.shard_ranges([5], 2) in ([(0, 1), (1, 0)], [(0, 0), (0, 1)])
    r = shard.shard_ranges([1, 1, 1], 5)                     # more ranks than subgrids
    assert sum(c for _, c in r) == 3 and all(c >= 0 for _, c in r)
    with pytest.raises(ValueError):
        shard.shard_ranges([1, 2], 0)

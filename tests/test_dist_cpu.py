"""Multi-rank paths of bench.py on the CPU (gloo, world size 2).

The gridder's work shards by job (each rank is an independent replica with
no data-path collective), so the only cross-rank steps are the barrier around
the timed region and the reductions that turn per-rank timings into the
whole-job figure: units summed over ranks, time the maximum over ranks.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(impl="reference")
    w, r, _ = bench.dist_setup(args)
    try:
        bench.barrier(w)
        # rank r processed (r + 1) * 1000 units in (r + 1) * 0.5 s
        rate = bench.whole_job_rate(w, (r + 1) * 0.5, (r + 1) * 1000.0)
        mx = bench.max_over_ranks(w, float(r))
        sm = bench.sum_over_ranks(w, float(r + 1))
        out_q.put((r, w, rate, mx, sm))
    finally:
        import torch.distributed as dist
        dist.destroy_process_group()


def test_whole_job_rate_two_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for r, w, rate, mx, sm in res:
        assert w == 2
        assert rate == pytest.approx(3000.0 / 1.0)     # (1000 + 2000) units over the slower rank's 1.0 s
        assert mx == 1.0
        assert sm == 3.0


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(1, 2.0, 10.0) == 5.0


def test_reference_arm_under_torchrun_prints_one_line():
    # launched as the two-rank reference arm: rank 0 times the oracle, rank 1 exits without work
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--config", "tiny", "--steps", "1", "--warmup", "0", "--cpu-seconds", "0.3"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle"
    assert rec["e2e"]["h2d_bytes_per_step"] == 0

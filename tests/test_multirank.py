"""The multi-process host path of bench.py on CPU: two gloo ranks (replicas, no data-path collective).

Under torchrun every rank solves its own problems and only the timing is reduced (the slowest rank);
these tests run that host logic, and the reference arm's rank handling, without a GPU.
"""
import json
import os
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
        sizes, seeds = bench.batch_problems(rank, 16)
        allseeds = [None] * world
        dist.all_gather_object(allseeds, seeds)
        allsizes = [None] * world
        dist.all_gather_object(allsizes, sizes)
        value = bench.whole_job_value(1000.0, world, ms)
        out.put((rank, ms, allseeds, allsizes, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_keep_problems_apart():
    world, port = 2, 29517
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, allseeds, allsizes, value in res:
        assert ms == 15.0  # both ranks see the slowest rank's time
        assert value == pytest.approx(1000.0 * world / 15e-3)
        assert not set(allseeds[0]) & set(allseeds[1])  # disjoint problems per rank
        assert allsizes[0] != allsizes[1]  # sizes drawn per rank
        import bench
        assert all(s in bench.BATCH_SIZES for s in allsizes[0] + allsizes[1])


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.whole_job_value(2.0e6, 1, 1000.0) == pytest.approx(2.0e6)


def test_reference_arm_under_torchrun_prints_on_rank_0_only(tmp_path):
    # two ranks of the reference arm: rank 1 exits 0 without work, rank 0 times the oracle and prints one line
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", "--master-port=29519", os.path.join(ROOT, "bench.py"), "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--cells", "32"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0

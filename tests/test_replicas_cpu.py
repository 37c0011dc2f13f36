"""The bench's multi-GPU path runs one independent replica per GPU (the
step exchanges nothing between GPUs): the job time is the slowest rank's
(max over ranks) and the throughput counts every rank's cells.  Checked
with two gloo ranks on the CPU (no GPU needed)."""
import os
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    try:
        mx = bench.max_over_ranks(10.0 + 5.0 * rank, device="cpu")
        q.put((rank, mx, bench.job_throughput(world, 1_000_000, mx)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time_and_sum_the_cells():
    world, port = 2, 29531 + os.getpid() % 1000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    assert [g[1] for g in got] == [15.0, 15.0]
    # 2 ranks x 1e6 cells in 15 ms
    assert got[0][2] == pytest.approx(2 * 1_000_000 / 15e-3)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, device="cpu") == 7.5
    assert bench.job_throughput(1, 119_299_098, 0.38) == pytest.approx(119_299_098 / 0.38e-3)

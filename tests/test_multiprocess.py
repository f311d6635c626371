"""The host side of the multi-GPU benchmark path, run as two gloo ranks on the CPU: the step time
is the slowest rank's and the whole-job rate counts every rank's frames (weak scaling)."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench._dist()
        own_ms = 2.0 + 3.0 * rank          # rank 1 is the slower replica
        ms = bench.max_over_ranks(own_ms, dist, "cpu")
        dist.barrier()
        q.put((r, ws, local, ms, bench.whole_job_rate(ws, 1_000_000, ms)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for r, (rank, ws, local, ms, rate) in enumerate(out):
        assert rank == r and ws == 2 and local == r
        assert ms == 5.0                   # max(2, 5) on both ranks
        assert rate == pytest.approx(2 * 1_000_000 / 5e-3 / 1e6)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(1, 2_000_000, 4.0) == pytest.approx(500.0)

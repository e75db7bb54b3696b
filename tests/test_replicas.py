"""The multi-replica bench path on the CPU (world size 2, gloo): the work does not
shard -- each rank images its own copy of the workload -- so the only exchange
is the timing reduction (max over ranks) and the whole-job rate rank 0 reports."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, times, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (world, rank, rank)
        ms = bench.max_over_ranks(times[rank], dist, "cpu")
        out[rank] = (ms, bench.whole_job_rate(1000, 4, world, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate():
    world, times = 2, [12.5, 20.0]
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), times, out), nprocs=world, join=True)
    for rank in range(world):
        ms, rate = out[rank]
        assert ms == 20.0  # the slowest replica ends the job
        assert rate == pytest.approx(1000 * 4 * world / 0.020)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(7.0) == 7.0
    assert bench.whole_job_rate(5, 2, 1, 10.0) == pytest.approx(1000.0)

"""Host logic of bench.py's multi-GPU mode (replicas, no collective on the
data path), run as world-size-2 gloo process groups on the CPU: the timing is
the slowest rank's, the throughput counts every replica's tensor, and the
reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.slowest_ms(times[rank], world, "cpu")
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("times", [(2.5, 3.75), (9.0, 1.0)])
def test_slowest_rank_sets_the_time(times):
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), times, out), nprocs=world, join=True)
        got = [out[r] for r in range(world)]
    assert got == [max(times)] * world


def test_whole_job_throughput_counts_every_replica():
    one = bench.job_gbs(1 << 30, 1, 2.0)
    assert one == pytest.approx((1 << 30) / 2e-3 / 1e9)
    assert bench.job_gbs(1 << 30, 4, 2.0) == pytest.approx(4 * one)
    assert bench.slowest_ms(3.0, 1, "cpu") == 3.0


def test_reference_arm_runs_on_rank_zero_only():
    class A:
        steps, warmup = 1, 0
    assert bench.run_reference(A, bench.WORKLOADS["c5"], rank=1, world=2) is None

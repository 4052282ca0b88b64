"""Host side of the partitioned sweep (tt_utv_sharded), on CPU with two gloo
ranks: each rank's slab of the whole tensor (mode 1 for the right-to-left
sweep, mode d for the left-to-right one), the all-reduce the library asks
for (a sum of FP64 partials that every rank receives equal) and the
all-gather (rank-ordered concatenation), through the same communicator
methods the GPU path calls."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import paper_2501_07904_gb300 as tu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        comm = tu.TorchDistComm(device="cpu")
        assert (comm.rank, comm.nranks) == (rank, world)
        A = torch.arange(4 * 3 * 6, dtype=torch.float32).reshape(4, 3, 6)
        rl = tu.slab(A, world, rank, "RL")
        lr = tu.slab(A, world, rank, "LR")
        # partial sums (FP64) of a per-rank Gram stand-in: every rank gets the total
        part = torch.full((5,), float(rank + 1), dtype=torch.float64) * torch.arange(5, dtype=torch.float64)
        comm.allreduce(part)
        # rank-ordered concatenation of byte blocks
        send = torch.full((8,), rank + 1, dtype=torch.uint8)
        recv = torch.empty(8 * world, dtype=torch.uint8)
        comm.allgather(send, recv)
        out[rank] = (rl.numpy().copy(), lr.numpy().copy(), part.numpy().copy(), recv.numpy().copy())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    A = np.arange(4 * 3 * 6, dtype=np.float32).reshape(4, 3, 6)
    rl = np.concatenate([out[r][0] for r in range(world)], axis=0)
    lr = np.concatenate([out[r][1] for r in range(world)], axis=2)
    assert np.array_equal(rl, A) and np.array_equal(lr, A)
    assert out[0][0].shape == (2, 3, 6) and out[0][1].shape == (4, 3, 3)
    total = sum((r + 1) * np.arange(5, dtype=np.float64) for r in range(world))
    for r in range(world):
        assert np.array_equal(out[r][2], total)
        assert list(out[r][3]) == [1] * 8 + [2] * 8


def test_slab_requires_equal_parts():
    with pytest.raises(ValueError):
        tu.slab(torch.zeros(5, 4), 2, 0, "RL")

"""The multi-GPU path of the benchmark is replicas only: each rank runs the
whole workload on its own GPU and the job reports every rank's Trotter steps
over the slowest rank's time.  Checked here with two gloo ranks on CPU."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = [2.0, 3.0][rank]
    t, v = bench.aggregate(elapsed, 500, dist, device="cpu")
    out[rank] = (t, v)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_take_max_time():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        t, v = out[r]
        assert t == 3.0
        assert v == pytest.approx(1000 / 3.0)


def test_single_rank():
    import bench

    t, v = bench.aggregate(4.0, 200, None)
    assert (t, v) == (4.0, 50.0)

"""The multi-GPU form of the bench is replicas only (the path shards without exchange): every rank
runs its own product and the slowest rank's time sets the whole-job rate.  The rank logic runs here
as two gloo processes on the CPU."""
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


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 10 + r ms for 3e9 units
        ms_max, value = bench.replica_throughput(10.0 + rank, 3e9, world, "cpu")
        dist.barrier()
        out[rank] = (ms_max, value)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank in range(world):
        ms_max, value = res[rank]
        assert ms_max == pytest.approx(11.0)
        # both replicas' units over the slowest rank's time
        assert value == pytest.approx(world * 3e9 / 11e-3 / 1e9)


def test_single_replica_needs_no_process_group():
    ms_max, value = bench.replica_throughput(4.0, 2e9, 1, "cpu")
    assert ms_max == 4.0 and value == pytest.approx(2e9 / 4e-3 / 1e9)

"""The multi-GPU path is independent replicas (no collective on the data
path); its host logic -- the max over ranks of the step time and the
whole-job rate -- is checked here with two gloo ranks on the CPU."""
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


def _worker(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    my_ms = 100.0 + 50.0 * rank  # the second replica is slower
    ms = bench.reduce_max(my_ms, world)
    out[rank] = bench.replica_rate(1000, ms, world)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    # both ranks see the max time (150 ms) and count both replicas' rays
    assert out[0] == pytest.approx(2 * 1000 / 0.150)
    assert out[1] == out[0]


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max(12.5, 1) == 12.5
    assert bench.replica_rate(500, 250.0, 1) == pytest.approx(2000.0)

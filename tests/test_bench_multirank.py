"""The replica (weak-scaling) aggregation of bench.py across ranks, on CPU
with the gloo backend and two processes."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_local = 2.0 if rank == 0 else 5.0
    value, t = bench.replica_throughput(t_local, 50, world, dist)
    out[rank] = (value, t)
    dist.destroy_process_group()


def test_replica_throughput_uses_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        res = dict(out)
    for r in range(world):
        value, t = res[r]
        assert t == pytest.approx(5.0)
        assert value == pytest.approx(world * 50 / 5.0)


def test_replica_throughput_single_rank():
    import bench
    assert bench.replica_throughput(4.0, 20, 1) == (5.0, 4.0)

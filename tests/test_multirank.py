"""The benchmark's multi-rank aggregation (independent replicas, one per GPU):
barrier-free max-over-ranks time and summed throughput, checked with two gloo
ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as td  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    td.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = [12.0, 30.0][rank]                       # rank 1 is the slowest
    n = [1000, 3000][rank]
    t_max, value = bench.aggregate(t, n, True)
    out[rank] = (t_max, value)
    td.barrier()
    td.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        t_max, value = out[r]
        assert t_max == 30.0
        assert value == pytest.approx(4000 / 30e-3)


def test_single_rank_aggregation():
    import bench
    assert bench.aggregate(10.0, 500, False) == (10.0, 500 / 10e-3)

"""Multi-GPU path of bench.py on CPU: replicas only, so the sole collective
is the all-reduce MAX of the timed seconds (world size 2, gloo, loopback);
every rank solves its own seeded system."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = 1.5 + rank  # rank 1 is the slowest
    out[rank] = (bench.max_over_ranks(local, world), bench.replica_seed(rank))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_distinct_systems():
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_rank, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    assert out[0][0] == out[1][0] == 2.5
    assert out[0][1] != out[1][1]


def test_single_rank_needs_no_collective():
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25

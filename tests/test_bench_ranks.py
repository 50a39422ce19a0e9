"""The multi-GPU path of bench.py (independent replicas, one process per GPU): its
whole-job aggregation -- time = max over ranks, flops = sum -- checked with two gloo ranks
on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    t, f = bench.aggregate_ranks(1.0 + rank, 10.0 * (rank + 1), "cpu")
    out[rank] = (t, f)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1] == (2.0, 30.0)


def test_aggregation_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(1.5, 7.0, "cpu") == (1.5, 7.0)

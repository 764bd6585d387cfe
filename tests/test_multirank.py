"""Weak-scaling aggregation across ranks, on CPU with two gloo ranks.

bench.py under torchrun gives every rank its own seeded scene of the same
size and reports sum(fragments) / max(time); this checks that reduction and
that the per-rank scenes differ, without a GPU.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        frags = 1000 * (rank + 1)
        ms = 2.0 + rank
        out[rank] = bench.aggregate(frags, ms, dist)
        w = bench.workload("spheres", rank)
        out[10 + rank] = float(w.scene.pos.sum())
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1] == (3000, 3.0)
    assert out[10] != out[11]  # each rank builds a different seeded scene

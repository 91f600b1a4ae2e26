"""The multi-rank (replica) aggregation of bench.py on CPU: two gloo ranks,
times take the maximum over ranks and flops the sum."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: ms = 10 + r, flops = 100 * (r + 1), e2e time 1 + r, e2e flops 7
        res = bench.aggregate_ranks(10.0 + rank, 100.0 * (rank + 1), 1.0 + rank, 7.0, world, "cpu")
        out[rank] = res
    finally:
        dist.destroy_process_group()


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        for r in range(world):
            assert out[r] == (11.0, 300.0, 2.0, 14.0)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(3.0, 4.0, 5.0, 6.0, 1, "cpu") == (3.0, 4.0, 5.0, 6.0)

"""The multi-GPU mode of bench.py is N independent replicas (one process per GPU,
each embedding its own copy of the workload); its only collective is the reduction
of the timed result: the slowest rank's time and the sum of all ranks' units.  This
runs that reduction with two gloo ranks on the CPU."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms, units = bench.reduce_over_ranks(dist, 10.0 + 5.0 * rank, 1000.0 * (rank + 1), "cpu")
        out[rank] = (ms, units)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_reduce_to_slowest_time_and_total_units():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    assert dict(out) == {0: (15.0, 3000.0), 1: (15.0, 3000.0)}

"""Host logic of the multi-GPU bench path (replicas, weak scaling), run as two gloo ranks
on the CPU: every rank sees the slowest rank's time, and the aggregate throughput is the
cells of all replicas over that time. (The GPU path is the same code with NCCL.)"""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [3.0, 5.0][rank]
    m = bench.max_over_ranks(ms)
    out[rank] = (m, bench.aggregate_mlups(256 ** 3, m, world))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_aggregate_two_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    assert out[0][0] == out[1][0] == 5.0
    assert out[0][1] == pytest.approx(2 * 256 ** 3 / 5e-3 / 1e6)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(4.25) == 4.25
    assert bench.aggregate_mlups(1000, 1.0, 1) == pytest.approx(1.0)

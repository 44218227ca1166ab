"""The multi-process (one rank per GPU, replicas) bookkeeping of bench.py on CPU: two gloo ranks
agree on the slowest rank's timed region, report whole-job throughput from it, and only rank 0
runs the oracle reference arm."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    got = bench.max_over_ranks(ms, dist, torch.device("cpu"))
    out[rank] = (got, bench.replica_throughput(world, 40, got))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_rank():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        got, thr = out[r]
        assert got == 150.0
        assert thr == pytest.approx(world * 40 / 0.150)


def test_single_process_keeps_its_own_time():
    assert bench.max_over_ranks(12.5, None, None) == 12.5
    assert bench.replica_throughput(1, 10, 12.5) == pytest.approx(800.0)


def test_reference_arm_runs_on_rank_zero_only():
    class Args:
        workload = "order3-50-r5"
    assert bench.reference_main(Args(), rank=1, world=2) is None  # returns before any work

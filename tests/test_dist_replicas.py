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


def test_reference_arm_prints_the_contract_line():
    """Rank 0 of the reference arm (the CPU FP64 oracle) prints one JSON line with the contract's
    keys; its step time and its throughput describe the same step (one sweep)."""
    import json
    import subprocess

    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--workload", "order3-50-r5"], capture_output=True, text=True,
                         timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "sweeps/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and abs(d["value"] * d["ms_per_step"] - 1000.0) <= 1e-6 * 1000.0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0

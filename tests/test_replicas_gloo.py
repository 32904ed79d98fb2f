"""CPU checks of bench.py's multi-rank (replica) path with two gloo ranks: the
timed region and the end-to-end time are the slowest rank's on every rank, the
whole-job throughput counts every rank's replica, and the reference arm prints from
rank 0 only."""
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
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms, e2e = bench.slowest_rank(10.0 * (rank + 1), 1.5 + rank, world, "cpu")
        out[rank] = (ms, e2e, bench.replica_throughput(1000, 5, world, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_slowest_rank_and_whole_job_throughput():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1]
    ms, e2e, value = out[0]
    assert ms == 20.0 and e2e == 2.5
    assert value == pytest.approx(1000 * 5 * 2 / 0.020)


def test_reference_arm_prints_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, gpus = 1, 0, 2
    bench.run_reference(A(), rank=1)
    assert capsys.readouterr().out == ""

"""The multi-rank bench path on CPU (gloo, world size 2): replicas, the
job's time is the slowest rank's and its throughput counts every rank's
decompositions; the reference arm does its work on rank 0 only."""
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
    import bench
    ms = 100.0 + 25.0 * rank                       # rank 1 is the slow one
    mx = bench.max_over_ranks(ms, world, "cpu")
    out[rank] = (mx, bench.replica_throughput(4, world, mx))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_time_and_job_throughput():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        mx, value = out[r]
        assert mx == 125.0
        assert value == pytest.approx(world * 4 / 0.125)


def test_reference_arm_only_on_rank_zero(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    assert bench.run_reference(bench.parse()) == 0
    assert capsys.readouterr().out == ""

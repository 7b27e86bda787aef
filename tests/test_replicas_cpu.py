"""The N > 1 path (independent replicas, one process per GPU) on CPU with gloo, world size 2:
the whole-job throughput is all ranks' units over the slowest rank's time on every rank, and
the reference arm's non-zero ranks exit without work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1912_06636_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, units, ms, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        value, slowest, total = replicas.aggregate(units[rank], ms[rank])
        out[rank] = (value, slowest, total)
    finally:
        dist.destroy_process_group()


def test_aggregate_two_ranks():
    world = 2
    units, ms = [1000.0, 3000.0], [250.0, 400.0]
    with mp.get_context("spawn").Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, _free_port(), units, ms, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        value, slowest, total = res[r]
        assert slowest == 400.0 and total == 4000.0
        assert value == pytest.approx(4000.0 / 0.4)


def test_aggregate_single_process():
    assert replicas.aggregate(500.0, 250.0) == (2000.0, 250.0, 500.0)


def test_reference_arm_other_ranks_exit(monkeypatch, capsys):
    import sys

    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    assert bench.run_reference(bench.parse()) is None  # rank 1: no work
    assert capsys.readouterr().out == ""               # and no line

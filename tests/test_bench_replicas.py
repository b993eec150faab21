"""The replica path of bench.py on CPU: two gloo ranks reduce their times with the helper the
bench uses (max over ranks) and form the whole-job value from the slowest rank; the reference
arm does no work and prints nothing on ranks other than 0."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    times = [10.0 + rank, 5.0 - rank]  # per-rank step and solve times (ms)
    tmax, smax = bench.replica_max(dist, times, "cpu")
    out[rank] = (tmax, smax, bench.whole_job_value(world, 1000, 4, smax))
    dist.destroy_process_group()


def test_replica_max_and_whole_job_value_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        tmax, smax, value = out[r]
        assert tmax == 11.0 and smax == 5.0
        assert value == pytest.approx(world * 1000 * 4 / 5e-3)


def test_replica_max_without_a_process_group():
    import bench
    assert bench.replica_max(None, [3.0, 4.0], "cpu") == [3.0, 4.0]


def test_reference_arm_is_silent_on_other_ranks(capsys, monkeypatch):
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(argparse.Namespace(steps=1, warmup=0))
    assert capsys.readouterr().out == ""

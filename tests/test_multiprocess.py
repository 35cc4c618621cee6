"""The multi-rank path of bench.py on CPU: two gloo ranks (127.0.0.1) take the
maximum of their timings, and the whole-job throughput of the replicas is
computed from the slowest rank.  The reference arm does nothing on rank > 0."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        times = [10.0 + rank, 5.0 * (world - rank)]  # rank 1 is slower on the first, rank 0 on the second
        got = bench.reduce_max(times, dist, device="cpu")
        out[rank] = got
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == [11.0, 10.0]


def test_job_throughput_of_replicas():
    sys.path.insert(0, ROOT)
    import bench
    # 2 replicas of 4.19 M cells, 100 steps each, slowest rank 20 ms
    assert bench.job_mlups(2, 4194304, 100, 20.0) == pytest.approx(2 * 4194304 * 100 / 0.020 / 1e6)
    assert bench.reduce_max([1.5, 2.5]) == [1.5, 2.5]


def test_reference_arm_is_silent_on_other_ranks(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup, gpus = 1, 0, 2

    bench.run_reference(Args())
    assert capsys.readouterr().out == ""

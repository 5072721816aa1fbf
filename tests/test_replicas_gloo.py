"""The N-GPU bench path on the host: N replicas each solve their own copy of
the workload, and the whole-job rate is N x steps over the slowest rank's time
(max over ranks), with no collective on the data path. Two gloo ranks on CPU."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 2 + r seconds for 5 solves
        rate, smax = bench.job_rate(2.0 + rank, 5, world)
        out[rank] = (rate, smax)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_rate_is_max_over_ranks_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    for r in range(world):
        rate, smax = res[r]
        assert smax == pytest.approx(3.0)
        assert rate == pytest.approx(world * 5 / 3.0)


def test_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    rate, smax = bench.job_rate(0.5, 10, 1)
    assert smax == 0.5 and rate == pytest.approx(20.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun only rank 0 times the oracle; the other ranks exit without work."""
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    bench.reference_arm(argparse.Namespace(steps=1, warmup=3, ref_iters=1))
    assert capsys.readouterr().out == ""

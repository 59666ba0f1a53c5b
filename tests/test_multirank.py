"""The N > 1 path of bench.py (independent replicas, one per rank): the timing
of the job is the slowest rank's, and the whole-job value counts every rank's
units.  Run as two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seconds = [0.5, 0.8][rank]          # rank 1 is the slower replica
    t = bench.max_over_ranks(seconds, dist, device="cpu")
    v = bench.job_value(1_000_000, world, t)
    dist.barrier()
    out[rank] = (t, v)
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_count_all_units():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        t, v = out[r]
        assert t == 0.8
        assert v == pytest.approx(2 * 1_000_000 / 0.8 / 1e6)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import argparse

    import bench
    args = argparse.Namespace(workload="2d", warmup=0, steps=1, gpus=2)
    bench.reference_arm(args, rank=1)
    assert capsys.readouterr().out == ""

"""The multi-GPU path of bench.py is replicas only: every rank decomposes its
own matrix, the job time is the max over ranks, and the reference arm runs on
rank 0 alone.  These checks run that host logic as two gloo ranks on the CPU."""
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


def _rank_main(rank, world, port, local_ms, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_max = bench.replica_max(local_ms[rank], dist, "cpu")
        out[rank] = (t_max, bench.replica_value(world, 10, t_max))
    finally:
        dist.destroy_process_group()


def test_replica_max_and_value_two_ranks():
    world, port = 2, _free_port()
    local_ms = [12.5, 20.0]
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, port, local_ms, out), nprocs=world,
                           start_method="spawn", join=True)
        res = dict(out)
    for r in range(world):
        t_max, value = res[r]
        assert t_max == 20.0                       # the slowest rank sets the job time
        assert value == pytest.approx(2 * 10 / 0.020)   # units of all ranks / that time


def test_single_process_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_max(7.25) == 7.25
    assert bench.replica_value(1, 4, 2.0) == pytest.approx(2000.0)


def test_reference_arm_other_ranks_do_no_work(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    import argparse
    bench.run_reference(argparse.Namespace(gpus=2, cpu_seconds=0.0))
    assert capsys.readouterr().out == ""

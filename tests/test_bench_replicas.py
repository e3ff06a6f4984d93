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


def test_clock_samples_kept_inside_the_timed_region(tmp_path, monkeypatch):
    # the sampler's lines carry timestamps; only those inside [start, stop]
    # count, and a region shorter than the interval reports its neighbours
    sys.path.insert(0, ROOT)
    import bench
    from datetime import datetime

    def line(ts, sm, reason="Not Active"):
        stamp = datetime.fromtimestamp(ts).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return "%s, 0, %d, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, %s\n" % (
            stamp, sm, reason)

    class FakeProc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            pass

    t0 = 1.8e9
    for lines, begin, end, want in (
            ([line(t0 - 0.02, 1500), line(t0 + 0.01, 2070), line(t0 + 0.03, 2000),
              line(t0 + 0.06, 1400, "Active")], t0, t0 + 0.04,
             {"sm_mhz": 2035.0, "samples": 2, "reasons": []}),
            ([line(t0 - 0.02, 1980), line(t0 + 0.02, 2070, "Active")], t0, t0 + 0.005,
             {"sm_mhz": 2025.0, "samples": 2, "reasons": ["sw_power_cap"]})):
        c = bench.Clocks(0)
        c.path = str(tmp_path / "clk.csv")
        with open(c.path, "w") as f:
            f.writelines(lines)
        c.proc, c.begin = FakeProc(), begin
        monkeypatch.setattr(bench.time, "time", lambda: end)
        monkeypatch.setattr(bench.time, "sleep", lambda s: None)
        got = c.stop()
        for k, v in want.items():
            assert got[k] == v, (k, got)


def test_one_core_cpu_baseline_runs_the_oracle_single_threaded():
    # the bench's 1-core oracle leg: a child process with every BLAS/OpenMP
    # pool held to one thread, at least one whole decomposition
    sys.path.insert(0, ROOT)
    import bench
    out = bench.one_core_oracle_rate(bench.WORKLOAD, 0.0)
    assert out["cores"] == 1 and out["kind"] == "oracle"
    assert out["value"] is not None and out["value"] > 0, out


def test_refined_pinv_flop_count_follows_the_shapes():
    sys.path.insert(0, ROOT)
    import bench
    w = {"c": 200, "r": 200, "rank_cap": 50}
    r = c = 200
    k = 50
    # float-float quaternion multiply-adds at three iterations: the first
    # iteration's X = W Z' and solves, two full iterations (Z, X, M, E, M',
    # the norm product, the solves), the ending (solves, E2, V, U); the FP32
    # products (Y0, the first Z and M, every G', G1 and G2) at 16/188 of one
    solves = (2 * c + r) * k * k / 2
    first = r * c * k + solves
    per_iter = 2 * r * c * k + r * k * k + c * k * k + k ** 3 + c * k * k + solves
    final = (r + c) * k * k + r * k * k + c * k * k + c * r * k
    fp32 = 2 * r * c * k + r * k * k + 3 * c * k * k / 2 + r * k * k
    expect = 32 * (first + 2 * per_iter + final + fp32 * 16.0 / 188)
    assert abs(bench.pinv_flops(w, "refined", 3) - expect) < 1e-6 * expect
    assert bench.pinv_flops(w, "refined", 4) > bench.pinv_flops(w, "refined", 3)


def test_stream_defaults(monkeypatch):
    # one stream with the FP64 Jacobi core (its own grid covers every SM),
    # eight otherwise; never more streams than the timed steps
    sys.path.insert(0, ROOT)
    import bench
    for argv, pinv, streams in ((["--workload", "color4096_smooth100"], "jacobi", 1),
                                ([], "refined", 8),
                                (["--pinv", "jacobi"], "jacobi", 1),
                                (["--streams", "4"], "refined", 4)):
        monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
        a = bench.parse()
        assert (a.pinv, a.streams) == (pinv, streams)


def test_stream_count_fills_whole_waves():
    sys.path.insert(0, ROOT)
    import bench
    # the default count divides the K steps into full waves where it can
    assert bench.stream_count(8, 200, True) == 8
    assert bench.stream_count(8, 20, True) == 5
    assert bench.stream_count(8, 11, True) == 6
    assert bench.stream_count(8, 3, True) == 3
    assert bench.stream_count(1, 20, True) == 1
    # an explicit count is kept, capped at K
    assert bench.stream_count(8, 20, False) == 8
    assert bench.stream_count(8, 3, False) == 3
    for K in range(1, 64):
        n = bench.stream_count(8, K, True)
        assert 1 <= n <= min(8, K)
        assert -(-K // n) * n <= -(-K // min(8, K)) * min(8, K)


def test_timed_repeats_releases_the_streams_together():
    # with several streams, every repeat puts a device sleep before its start
    # event on the launching stream (sized from the previous repeat's enqueue
    # time, outside the timed region) and the streams wait for that event;
    # with one stream there is no sleep
    sys.path.insert(0, ROOT)
    import bench
    calls = []

    class Ev:
        def __init__(self, enable_timing=False):
            pass

        def record(self, st=None):
            calls.append(("record", st))

        def elapsed_time(self, other):
            return 400.0

    class St:
        def wait_event(self, e):
            calls.append(("wait", self))

    class Cur:
        def wait_event(self, e):
            calls.append(("join",))

    cur = Cur()

    class Cuda:
        Event = Ev

        def synchronize(self):
            calls.append(("sync",))

        def current_stream(self):
            return cur

        def _sleep(self, cycles):
            calls.append(("sleep", cycles))

    class FakeTorch:
        cuda = Cuda()

    def run_once():
        calls.append(("run",))

    streams = [St(), St()]
    times = bench.timed_repeats(FakeTorch, run_once, streams, 1.0, sm_mhz=2000.0)
    assert times == [400.0] * 3
    sleeps = [c for c in calls if c[0] == "sleep"]
    assert len(sleeps) == 3
    assert sleeps[0][1] == int(5.0 * 1e3 * 2000.0)          # the first repeat's guess
    assert all(s[1] < sleeps[0][1] for s in sleeps[1:])      # then the measured enqueue time
    for i, c in enumerate(calls):
        if c[0] == "sleep":   # sleep, start event, both streams wait, then the steps
            assert calls[i + 1] == ("record", cur)
            assert [x[0] for x in calls[i + 2:i + 5]] == ["wait", "wait", "run"]
    calls.clear()
    assert bench.timed_repeats(FakeTorch, run_once, [], 1.0) == [400.0] * 3
    assert not [c for c in calls if c[0] == "sleep"]


def test_jacobi_pinv_flop_count_follows_the_shapes():
    # per column pair of the round-robin order (n_c/2 pairs in each of n_c - 1
    # steps for even n_c): the two squared norms (8 flops per entry each) and
    # conj(x) y (32) over the n_r rows of G, then q w (32) and the two
    # combinations (16) over the rows of G and of V (n_r + n_c)
    sys.path.insert(0, ROOT)
    import bench
    for r, c, sweeps in ((200, 200, 16), (500, 500, 30), (120, 90, 9), (91, 91, 5)):
        nr, nc = max(r, c), min(r, c)
        N = nc + nc % 2
        pairs = N // 2 * (N - 1)
        expect = sweeps * pairs * (48 * nr + 48 * (nr + nc))
        got = bench.pinv_flops({"c": c, "r": r, "rank_cap": 10}, "jacobi", sweeps)
        assert got == expect, (r, c, got, expect)
    # the colour field's 500 x 500 at 30 sweeps: 2.69e11
    assert abs(bench.pinv_flops({"c": 500, "r": 500, "rank_cap": 100}, "jacobi", 30)
               - 2.694e11) < 1e9

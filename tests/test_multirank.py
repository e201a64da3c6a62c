"""The multi-GPU path of bench.py on CPU ranks (gloo, world size 2).

Bands are independent, so N GPUs run N replicas with no data-path
collective: each rank builds its own seeded inputs, times its own steps
between barriers, and the job's time is the maximum over the ranks.  These
tests run that host logic as two gloo processes on 127.0.0.1.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, queue):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_info()
        ms = 10.0 + 5.0 * rank                 # rank 1 is the slow one
        job_ms = bench.max_over_ranks(torch, dist, ms)
        rate = bench.job_rate(ws, 1000, 20, job_ms)
        noise = bench.band_inputs(bench.WORKLOADS["tersoff_graphite_hexdiamond_576"],
                                  seed=2510 + r)["noise"]
        queue.put((rank, ws, r, job_ms, rate, float(noise[0, 0, 0])))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_time():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(queue.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, r, job_ms, rate, _ in out:
        assert ws == 2 and r == rank
        assert job_ms == 15.0                    # max over ranks
        assert rate == pytest.approx(2 * 1000 * 20 / 0.015)
    # each replica draws its own seeded interior jitter
    assert out[0][5] != out[1][5]


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"steps": 1, "warmup": 3, "gpus": 2})()
    assert bench.run_reference(args, "tersoff_graphite_hexdiamond_98304") == 0
    assert capsys.readouterr().out == ""

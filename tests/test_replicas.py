"""Multi-process path of the benchmark (replicas only: every rank runs its own replica, the
job's time is the slowest rank's, throughput counts the units of all ranks), run as two gloo
ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(times[rank], tdist, world, torch.device("cpu"))
        v = bench.job_throughput(world, 60, ms)
        q.put((rank, ms, v))
    finally:
        tdist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank_and_all_units():
    world, times = 2, [250.0, 400.0]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, world, port, times, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, v in out:
        assert ms == 400.0
        assert abs(v - 2 * 60 / 0.4) < 1e-9


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(123.0, None, 1, None) == 123.0
    assert bench.job_throughput(1, 10, 1000.0) == 10.0

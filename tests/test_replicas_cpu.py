"""The benchmark's multi-rank host logic on CPU ranks (gloo): replicas only --
each rank processes its own copy of the workload, the job time is the
slowest rank's, and the whole-job throughput counts every rank's records."""
import os
import socket

import pytest


def _worker(rank, world, port, ms, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(ms[rank], world, "cpu")
    out.put((rank, t, bench.job_throughput(world, 10**9, 10, t)))
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_replicas_take_the_slowest_rank():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    ms = [400.0, 500.0]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, ms, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [500.0, 500.0]
    assert res[0][2] == pytest.approx(2 * 10**9 * 10 / 0.5 / 1e9)


def test_single_rank_is_its_own_time():
    import bench
    assert bench.max_over_ranks(123.0, 1, "cpu") == 123.0
    assert bench.job_throughput(1, 10**9, 10, 500.0) == pytest.approx(20.0)

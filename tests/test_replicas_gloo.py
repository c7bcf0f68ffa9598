"""The N > 1 path of bench.py (replicas only: every rank runs its own copy of
the workload, the job's time is the slowest rank's, its work the sum of all
ranks'), run as two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t = bench.max_over_ranks(10.0 + 7.5 * rank, dist, "cpu")  # rank 1 is the slow replica
        rate = bench.whole_job_rate(1000.0, world, t)
        q.put((rank, t, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_time_and_sum_the_work():
    import torch.multiprocessing as mp
    pytest.importorskip("torch.distributed")
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    for rank, t, rate in out:
        assert t == 17.5  # every rank sees the slowest replica's time
        assert rate == pytest.approx(2 * 1000.0 / 17.5)


def test_single_process_needs_no_collective():
    import bench
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
    assert bench.whole_job_rate(100.0, 1, 2.0) == 50.0

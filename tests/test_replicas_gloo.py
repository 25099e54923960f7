"""The N > 1 bench path (replicas only): two gloo ranks on the CPU agree on
the slowest rank's time and on the whole-job value."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    total, value = bench.job_time_and_value(100.0 + 50.0 * rank, 1_000_000, 3, world, "cpu")
    q.put((rank, total, value))
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, value in out:
        assert total == pytest.approx(150.0)
        assert value == pytest.approx(2 * 1_000_000 * 3 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    total, value = bench.job_time_and_value(80.0, 500, 4, 1, "cpu")
    assert total == 80.0 and value == pytest.approx(500 * 4 / 0.08)

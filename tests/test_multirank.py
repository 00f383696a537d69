"""The multi-GPU path of bench.py is replicas only (the solve does not shard): every
rank solves its own problem, the step time is the slowest rank's, and the job's
seconds per solve is that time over the number of replicas.  This checks that
reduction with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [12.5, 40.0][rank]
    ms_max = bench.max_over_ranks(local_ms, dist, "cpu")
    q.put((rank, ms_max, bench.job_seconds_per_solve(ms_max, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, sec in out:
        assert ms_max == 40.0
        assert sec == pytest.approx(40.0 / 1000.0 / world)


def test_single_rank_without_process_group():
    import bench
    assert bench.max_over_ranks(7.0, None, "cpu") == 7.0
    assert bench.job_seconds_per_solve(7.0, 1) == pytest.approx(0.007)

"""The multi-rank logic of bench.py (replicas: one workload copy per rank, the
job time is the slowest rank's) on two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [12.5, 30.0][rank]
    mx = bench.max_over_ranks(local, world)
    val = bench.job_value(world, 1000, 150, mx)
    out.put((rank, mx, val))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, mx, val in res:
        assert mx == 30.0                       # slowest rank
        assert val == pytest.approx(2 * 1000 * 150 / 0.030)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(7.0, 1) == 7.0
    assert bench.job_value(1, 10, 3, 1000.0) == pytest.approx(30.0)

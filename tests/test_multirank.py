"""The multi-rank host logic of bench.py on CPU (gloo, world size 2).

The coupling step shards as independent replicas: every rank couples its own
workload, the job time is the maximum over ranks, and the whole-job rate is
world * nodes / that time.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    times = [1.0 + rank, 5.0 - rank]          # rank 0: (1, 5); rank 1: (2, 4)
    t = bench.max_over_ranks(times, "cpu", dist)
    out[rank] = (t, bench.job_throughput(1000, world, t[0]))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_gloo_world2():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        t, rate = out[r]
        assert t == [2.0, 5.0]
        assert rate == pytest.approx(2 * 1000 / 2e-3)


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks([3.0, 4.0], "cpu", None) == [3.0, 4.0]
    assert bench.job_throughput(10, 1, 2.0) == pytest.approx(5000.0)

"""Replica timing of bench.py over world_size 2 (gloo on CPU): the whole-job rate counts
every rank's units over the slowest rank's time, with no collective on the data path."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 1000.0 if rank == 0 else 4000.0       # rank 1 is the slow one
    value, ms_max = bench.job_rate(ms_local, 6, world, "cpu")
    out.put((rank, value, ms_max))
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_takes_slowest_rank_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, value, ms_max in res:
        assert ms_max == 4000.0                      # max over ranks
        assert value == pytest.approx(12 / 4.0)      # 6 units x 2 ranks / 4 s


def test_job_rate_single_rank():
    import bench
    value, ms_max = bench.job_rate(500.0, 3, 1, "cpu")
    assert ms_max == 500.0 and value == pytest.approx(6.0)

"""The replica path of bench.py (one process per GPU, no data exchange) on
CPU: two gloo ranks agree on the job time (the slowest rank) and on the
whole-job throughput (all ranks' units over that time)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 10.0 + 5.0 * rank              # rank 1 is the slow one
        ms = bench.job_time(ms_local, dist, torch.device("cpu"))
        out[rank] = (ms, bench.job_value(1_000_000, world, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_job_time_and_value():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == pytest.approx(15.0)
    assert res[0][1] == res[1][1] == pytest.approx(2 * 1_000_000 / 0.015)


def test_single_process():
    assert bench.job_time(12.5) == 12.5
    assert bench.job_value(600, 1, 2.0) == pytest.approx(300_000)

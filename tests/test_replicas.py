"""The replicas path of the benchmark (N > 1 processes): job rate from the slowest
rank, with two gloo ranks on the CPU."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, local_ms, out):
    import torch.distributed as dist
    from paper_2601_09417_gb300.replicas import job_rate
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = job_rate(local_ms[rank], 100)
    finally:
        dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank():
    port = _free_port()
    local_ms = [400.0, 500.0]
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, port, local_ms, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        total, rate = res[rank]
        assert total == pytest.approx(500.0)
        assert rate == pytest.approx(2 * 100 / 0.5)


def test_job_rate_single_process():
    from paper_2601_09417_gb300.replicas import job_rate
    total, rate = job_rate(250.0, 50)
    assert total == 250.0 and rate == pytest.approx(200.0)

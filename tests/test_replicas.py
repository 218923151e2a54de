"""The N > 1 path of bench.py (replicas: one independent evaluation per rank, no data-path
collective): the time is the maximum over ranks and the throughput counts every rank's pixels.
Two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank            # rank 1 is the slower replica
        worst = bench.max_over_ranks(ms, dist, torch.device("cpu"))
        value = bench.whole_job_mpx_s(world, 3024, 4032, 10, worst / 1e3)
        out[rank] = (worst, value)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    assert out[0] == out[1]
    worst, value = out[0]
    assert worst == 150.0
    assert value == pytest.approx(2 * 3024 * 4032 * 10 / 0.15 / 1e6)


def test_single_process_is_the_identity():
    assert bench.max_over_ranks(7.5, None, None) == 7.5
    assert bench.whole_job_mpx_s(1, 1000, 1000, 2, 0.5) == pytest.approx(4.0)

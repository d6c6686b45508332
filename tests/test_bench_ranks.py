"""The multi-rank bookkeeping of bench.py on CPU ranks (gloo, world size 2):
the job time is the slowest rank's and the throughput counts every rank's
cells; replicas exchange nothing but that one timing reduction."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        el = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
        out[rank] = (el, bench.replica_throughput(4096 * 4096, 2000, 10, world, el))
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_reduction():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0][0] == out[1][0] == 15.0
    expect = 4096 * 4096 * 2000 * 10 * 2 / 0.015 / 1e9
    assert abs(out[0][1] - expect) < 1e-9 * expect and out[0][1] == out[1][1]


def test_single_rank_is_identity():
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.replica_throughput(100, 10, 2, 1, 1000.0) == 100 * 10 * 2 / 1.0 / 1e9

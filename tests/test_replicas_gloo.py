"""The multi-GPU form of the bench is replicas only: every rank factors its own
copy of the workload, the job's time is the slowest rank's (max over the
process group) and the throughput sums the ranks' work.  Checked with two
gloo ranks on the CPU."""
from __future__ import annotations

import importlib.util
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        bench = _bench()
        flops = 6.0e11
        sec_local = 1.0 + rank          # rank 1 is the slow one
        value, sec_max = bench.aggregate(world, flops, sec_local, dist, torch.device("cpu"))
        out[rank] = (value, sec_max)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replicas_max_over_ranks_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        value, sec_max = out[r]
        assert sec_max == pytest.approx(2.0)
        assert value == pytest.approx(world * 6.0e11 / 2.0 / 1e9)


def test_single_rank_aggregate_is_local():
    bench = _bench()
    value, sec = bench.aggregate(1, 3.0e11, 0.5)
    assert sec == 0.5 and value == pytest.approx(600.0)

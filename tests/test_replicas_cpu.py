"""The N > 1 benchmark path on CPU: gloo ranks as independent replicas (no GPU).

Each rank times its own replica; the job's time is the maximum over ranks and
its throughput counts every rank's sweeps.  No data-path collective exists.
"""
from __future__ import annotations

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 + 50.0 * rank  # rank 1 is the slow replica
        total = bench.combine_ranks(local_ms, dist)
        dist.barrier()
        out[rank] = (total, bench.job_value(1000, world, total))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replicas_take_max_time_and_sum_work(world):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        total, value = out[r]
        assert total == 150.0
        assert value == pytest.approx(world * 1000 / 0.150)


def test_single_rank_needs_no_process_group():
    assert bench.combine_ranks(12.5, None) == 12.5
    assert bench.job_value(10, 1, 1000.0) == pytest.approx(10.0)

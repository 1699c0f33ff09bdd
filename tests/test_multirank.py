"""The bench's multi-rank aggregation (replicas, one per rank) on CPU with gloo,
world size 2: the job time is the slowest rank's and the value counts every
rank's samples."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.job_ms(10.0 + 5.0 * rank, world, "cpu")
        out[rank] = (ms, bench.job_value(1000, 4, ms, world))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        ctx = mp.get_context("spawn")
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1] == (15.0, 2 * 1000 * 4 / 0.015)


def test_single_rank_is_identity():
    assert bench.job_ms(12.5, 1, "cpu") == 12.5
    assert bench.job_value(10, 2, 1000.0, 1) == pytest.approx(20.0)

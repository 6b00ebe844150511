"""Replica sharding across ranks, on CPU with the gloo backend (world size 2):
each rank runs its own walker (distinct seed, no data exchange) and the job's
throughput divides all ranks' work by the slowest rank's step time."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import inputs


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = [3.0, 5.0][rank]
        value, ms = bench.job_throughput(ms_local, world, 64 * 64, 96, dist, "cpu")
        w = bench.walker_of(rank)
        seed = inputs.workload_seed(4, w)
        out[rank] = (value, ms, w, seed)
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank_and_shard_walkers():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        value, ms, w, seed = res[rank]
        assert ms == 5.0
        assert value == pytest.approx(world * 64 * 64 * 96 / 5e-3 / 1e9)
    assert {res[r][2] for r in range(world)} == {0, 1}
    assert res[0][3] != res[1][3]


def test_single_rank_needs_no_collective():
    value, ms = bench.job_throughput(4.0, 1, 2048 * 2048, 96)
    assert ms == 4.0
    assert value == pytest.approx(2048 * 2048 * 96 / 4e-3 / 1e9)

"""Host logic of the multi-GPU path (independent replicas), on CPU: two gloo
ranks in separate processes exchange the job totals exactly as the GPU
ranks do over NCCL, and every rank gets its own problem."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import igdata
from paper_2507_14222_gb300 import replicas


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # Each rank's own synthetic problem, as bench.py draws it.
        w = igdata.tiny(replicas.replica_seed(1001, rank))
        units = float(w.train_codes.shape[0] * (rank + 1))
        elapsed = 10.0 + 5.0 * rank
        replicas.barrier()
        t, u = replicas.job_totals(elapsed, units)
        mine = list(replicas.assign(10, rank, world))
        out[rank] = (t, u, mine, int(w.train_codes.sum()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_job_totals_and_problem_assignment(world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world,
                           start_method="spawn", join=True)
        res = dict(out)
    n = igdata.tiny().train_codes.shape[0]
    for rank in range(world):
        t, u, mine, _ = res[rank]
        assert t == 10.0 + 5.0 * (world - 1)          # slowest rank
        assert u == float(n * sum(r + 1 for r in range(world)))
    # every item is taken once, in order
    assert sorted(i for r in range(world) for i in res[r][2]) == list(range(10))
    # the ranks' problems differ
    assert res[0][3] != res[1][3]


def test_single_process_totals_are_identity():
    assert not dist.is_initialized()
    assert replicas.job_totals(3.5, 7) == (3.5, 7.0)
    replicas.barrier()


def test_assign_partitions():
    for n in (0, 1, 5, 64, 65):
        for world in (1, 2, 3, 8):
            blocks = [replicas.assign(n, r, world) for r in range(world)]
            assert [i for b in blocks for i in b] == list(range(n))
            sizes = [len(b) for b in blocks]
            assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    with pytest.raises(ValueError):
        replicas.assign(4, 2, 2)


def test_replica_seeds_are_distinct_problems():
    seeds = [replicas.replica_seed(1002, r) for r in range(8)]
    assert seeds[0] == 1002 and len(set(seeds)) == 8
    a = igdata.tiny(replicas.replica_seed(1001, 0)).train_codes
    b = igdata.tiny(replicas.replica_seed(1001, 1)).train_codes
    assert a.shape == b.shape and not np.array_equal(a, b)

"""Multi-process (gloo, world size 2, CPU) tests of the replica bookkeeping
that bench.py uses for runs on several GPUs."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2003_13163_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = replicas.world()
        assert (w, r, lr) == (world, rank, rank)
        replicas.barrier()
        # rank r did (r+1)*10 gates in (r+1) seconds
        rate, tot, tmax = replicas.job_rate((rank + 1) * 10.0, float(rank + 1))
        out[rank] = (rate, tot, tmax, replicas.rank_seed(100, rank), tuple(replicas.seeds_for(0, 5, world, rank)))
    finally:
        dist.destroy_process_group()


def test_two_rank_job_rate_and_seeds():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        rate, tot, tmax, seed, seeds = out[r]
        assert tot == 30.0 and tmax == 2.0 and rate == 15.0
        assert seed == 100 + r
    assert out[0][4] == (0, 2, 4) and out[1][4] == (1, 3)


def test_single_process_defaults():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.job_rate(10.0, 2.0) == (5.0, 10.0, 2.0)

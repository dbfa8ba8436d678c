"""The multi-process path of bench.py on CPU: two gloo ranks.

With N GPUs the benchmark runs N independent replicas (the method does not
shard one lattice), one per rank, with distinct seeds, and reports the time
of the slowest rank.  These tests run that aggregation with the gloo backend
on the host (no GPU): max over ranks, distinct replica seeds, and the weak
scaling value formula.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 + 3.0 * rank)
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.replica_seed(rank))
    out[rank] = (ms, tuple(seeds))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_distinct_replicas():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 13.0
    seeds = res[0][1]
    assert len(set(seeds)) == world and seeds == res[1][1]


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.max_over_ranks(4.5) == 4.5
    assert bench.replica_seed(0) == bench.SEED_BENCH

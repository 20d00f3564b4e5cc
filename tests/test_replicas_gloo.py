"""The N > 1 bench path without a GPU: two gloo ranks on the CPU.  The path
shards nothing (replicas only): every rank maps its own stretch of street and
the job's time is the slowest rank's."""
import os
import socket

import pytest
import torch.multiprocessing as tmp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first = bench.replica_first_scan(rank)
        slowest = bench.max_over_ranks(10.0 + rank, world, torch.device("cpu"))
        firsts = [None] * world
        dist.all_gather_object(firsts, first)
        out[rank] = (slowest, firsts)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_disjoint_scans_and_the_slowest_time():
    ctx = tmp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        slowest, firsts = res[r]
        assert slowest == 11.0
        assert firsts == [0, 1000]
    # the stretches do not overlap for any sequence length the bench uses (<= 1000 scans)
    assert firsts[1] - firsts[0] >= 1000


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1, None) == 3.5

"""Host-side multi-rank logic of bench.py on CPU (gloo, world size 2).

Blocks are independent, so ranks need no data-path collective: each rank
takes its block range (the full batch under weak scaling, or a contiguous
share) and the ranks only agree on the slowest timed region.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = bench.shard_blocks(1003, rank, world, weak=False)
        weak = bench.shard_blocks(1003, rank, world, weak=True)
        slowest = bench.max_over_ranks(10.0 + rank, world, None)
        bench.barrier(world)
        q.put((rank, mine, weak, slowest))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, w0, s0), (r1, m1, w1, s1) = out
    # contiguous split covering 0..1002 exactly once
    assert m0 == (0, 502) and m1 == (502, 501)
    # weak scaling: every rank transforms the full batch
    assert w0 == w1 == (0, 1003)
    # max over ranks of the timed region
    assert s0 == s1 == 11.0


def test_single_rank_helpers():
    assert bench.shard_blocks(10, 0, 1, weak=False) == (0, 10)
    assert bench.max_over_ranks(3.5, 1) == 3.5

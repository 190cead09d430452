"""Rank plumbing of bench.py (replicas only) on the CPU: two gloo ranks initialise from the
environment, meet at the barrier and agree on the maximum of their timings."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench

    r, ws, dist = bench.dist_init()
    try:
        bench.barrier(dist)
        m = bench.max_over_ranks(10.0 + r, dist)
        out.put((r, ws, m))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, 2, 11.0), (1, 2, 11.0)]


def test_single_process_needs_no_group():
    import bench

    os.environ.pop("WORLD_SIZE", None)
    r, ws, dist = bench.dist_init()
    assert (r, ws, dist) == (0, 1, None)
    assert bench.max_over_ranks(3.5, dist) == 3.5

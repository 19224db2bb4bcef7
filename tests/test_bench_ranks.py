"""The multi-rank host logic of bench.py on two gloo ranks (CPU).

The path does not shard: each rank solves its own replica and the only
cross-rank steps are the barrier around the timed region and the maximum of
the ranks' times.  Two processes rendezvous on 127.0.0.1 with the gloo
backend (the one `--impl reference` uses), pass the barrier, and both must
receive the larger of their two times; the reference arm's second rank must
return at once, leaving the oracle sample to rank 0.
"""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import argparse

    import bench
    args = argparse.Namespace(impl="reference")
    w, r, _ = bench.dist_init(args)
    bench.barrier(w)
    m = bench.max_over_ranks(10.0 + r, w)
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((r, w, m))


def _reference_worker(rank, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                      LOCAL_RANK=str(rank))
    import argparse
    import time

    import bench
    args = argparse.Namespace(impl="reference")
    t0 = time.time()
    if rank == 1:
        bench.run_reference(args)  # joins the group and returns: rank 0 alone times the oracle
        w = 2
    else:
        w, _, _ = bench.dist_init(args)  # stands in for rank 0 (its oracle sample is not run here)
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((rank, time.time() - t0))


def _run(target, args_of_rank):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=args_of_rank(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    for p in procs:
        if p.is_alive():
            p.kill()
            pytest.fail("a gloo rank did not finish")
        assert p.exitcode == 0
    return sorted(q.get(timeout=10) for _ in range(2))


def test_two_gloo_ranks_share_the_slowest_time():
    got = _run(_worker, lambda r, port, q: (r, 2, port, q))
    assert got == [(0, 2, 11.0), (1, 2, 11.0)]


def test_reference_arm_second_rank_returns_without_work():
    got = _run(_reference_worker, lambda r, port, q: (r, port, q))
    assert [r for r, _ in got] == [0, 1]
    assert all(t < 60 for _, t in got)  # no oracle sample was run on either rank

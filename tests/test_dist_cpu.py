"""The multi-rank path of bench.py on CPU (gloo, world size 2): the path
shards without any data exchange ("replicas only"), so ranks meet only at
the barriers around the timed region and in the max-over-ranks of its
duration; the whole-job value counts every rank's units against the slowest
rank's time, and the reference arm runs on rank 0 alone."""
import argparse
import multiprocessing as mp
import os
import socket

import pytest

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    try:
        d = bench.Dist(world)
        d.barrier()
        slowest = d.max(10.0 + 5.0 * rank)              # per-rank timed region, ms
        rate = bench.replica_rate(d.world, 100.0, 3, slowest)
        args = argparse.Namespace(shape="64,64,16", warmup=0, steps=1)
        ref = bench.run_reference(args, d) if rank == 1 else "skipped"
        d.barrier()
        d.close()
        q.put((rank, d.world, slowest, rate, ref))
    except Exception as e:  # reported to the parent, which fails the test
        q.put((rank, "error", repr(e), None, None))


def test_two_ranks_barrier_max_and_aggregate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = {}
    try:
        for _ in range(world):
            rank, *rest = q.get(timeout=120)
            results[rank] = rest
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.terminate()
    assert sorted(results) == [0, 1]
    for rank, (w, slowest, rate, ref) in results.items():
        assert w == world, (rank, slowest)
        assert slowest == pytest.approx(15.0)             # max over ranks
        assert rate == pytest.approx(2 * 100.0 * 3 / 0.015)
    assert results[1][3] is None                           # reference arm: rank 0 only


def test_single_rank_needs_no_process_group():
    d = bench.Dist(1)
    assert d.world == 1 and d.pg is None
    d.barrier()
    assert d.max(3.5) == 3.5
    assert bench.replica_rate(1, 10.0, 2, 4.0) == pytest.approx(5000.0)
    d.close()

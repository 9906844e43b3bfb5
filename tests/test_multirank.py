"""The N > 1 path of bench.py on CPU: two gloo ranks (spawned processes, rendezvous on 127.0.0.1).

Queries shard by rank with no data exchange; the only collective is the
max-over-ranks reduction of the timed region, and the whole-job rate counts
every rank's queries over the slowest rank's time.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2103_14915_gb300 import inputs
        ws, r, local = bench.dist_env()
        g = inputs.grid(64, 64, 500, 100, seed=3, weights=(100, 10000))
        sets = bench.source_sets(g, r, nq=32)
        slowest = bench.max_over_ranks(10.0 * (r + 1), torch.device("cpu"))
        rate = bench.job_rate(100, ws, slowest)
        q.put((r, ws, local, [s.tolist() for s in sets], slowest, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_queries_and_reduce_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        out = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    (r0, ws0, l0, sets0, slow0, rate0), (r1, ws1, l1, sets1, slow1, rate1) = out
    assert (r0, r1) == (0, 1) and ws0 == ws1 == 2 and (l0, l1) == (0, 1)
    # max over ranks: rank 1 reported 20 ms, both see it; the rate counts both ranks' queries
    assert slow0 == slow1 == 20.0
    assert rate0 == rate1 == pytest.approx(100 * 2 / 0.020)
    # every rank draws its own seeded source sets (its shard of the job)
    assert len(sets0) == len(sets1) == 3
    for a, b in zip(sets0, sets1):
        assert len(a) == len(b) == 32 and len(set(a)) == 32 and a != b


def test_single_process_needs_no_group():
    import bench
    assert not dist.is_initialized()
    assert bench.max_over_ranks(7.5, torch.device("cpu")) == 7.5
    assert bench.job_rate(2048, 1, 500.0) == pytest.approx(4096.0)

"""Host-side logic that needs no GPU: serving admission and batching, and
the multi-rank aggregation of bench.py (world size 2 over gloo)."""
import collections
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2402_02044_b300.serve import QUERY, Admission, LatencyStats, Request, bucket, form_batch, request_bytes


def _req(n, k=10, d=8):
    return Request(QUERY, np.zeros((n, d), np.float32), k, nbytes=request_bytes(QUERY, n, d, k))


def test_admission_budget():
    a = Admission(1000)
    assert a.fits_ever(1000) and not a.fits_ever(1001)
    assert a.try_take(600) and not a.try_take(500) and a.try_take(400)
    a.give(600)
    assert a.used == 400 and a.try_take(600)


def test_form_batch_keeps_order_and_limits():
    q = collections.deque([_req(3), _req(5), _req(7), _req(1)])
    a = Admission(10 ** 9)
    b = form_batch(q, 10, a)
    assert [r.data.shape[0] for r in b] == [3, 5]          # 3 + 5 + 7 > 10
    assert [r.data.shape[0] for r in q] == [7, 1]
    b = form_batch(q, 10, a)
    assert [r.data.shape[0] for r in b] == [7, 1]
    # a request larger than the batch limit still goes, alone
    q = collections.deque([_req(40), _req(2)])
    assert [r.data.shape[0] for r in form_batch(q, 10, a)] == [40]


def test_form_batch_takes_only_accepted_heads():
    q = collections.deque([_req(3), _req(5), _req(2)])
    q[0].group = q[1].group = "open"
    a = Admission(10 ** 9)
    b = form_batch(q, 100, a, accept=lambda r: r.group == "open")
    assert [r.data.shape[0] for r in b] == [3, 5] and [r.data.shape[0] for r in q] == [2]
    assert form_batch(q, 100, a, accept=lambda r: r.group == "open") == []


def test_form_batch_respects_the_byte_budget():
    one = request_bytes(QUERY, 4, 8, 10)
    a = Admission(2 * one + 1)
    q = collections.deque([_req(4), _req(4), _req(4)])
    assert len(form_batch(q, 100, a)) == 2 and len(q) == 1
    assert form_batch(q, 100, a) == []                     # waits for bytes
    a.give(one)
    assert len(form_batch(q, 100, a)) == 1


def test_bucket_and_stats():
    assert [bucket(n) for n in (1, 2, 3, 16, 17, 4096)] == [1, 2, 4, 16, 32, 4096]
    s = LatencyStats()
    for i in range(100):
        s.add(0.0, (i + 1) * 1e-3, 2)
    out = s.summary()
    assert abs(out["p50_ms"] - 50.5) < 1e-6 and abs(out["p99_ms"] - 99.01) < 1e-6
    assert abs(out["qps"] - 2000.0) < 1e-6


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units, secs = bench.aggregate(100.0 * (rank + 1), 1.0 + rank, world)
    out[rank] = (units, secs)
    dist.destroy_process_group()


def test_bench_aggregates_units_and_slowest_rank_over_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
    assert all(p.exitcode == 0 for p in procs)
    assert out[0] == (300.0, 2.0) and out[1] == (300.0, 2.0)

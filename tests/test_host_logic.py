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


def test_fixed_point_query_error_bound():
    """The ID-gather first level scales the float32 query by a power of two,
    s = 2^(e - 30) with 2^e <= max|q| < 2^(e+1), rounds it once
    (Q = rint(q / s), |Q| < 2^31) and multiplies Q with the codes exactly.
    The change of <q, x^> (x^ = l + D c) is D sum_j (q_j - s Q_j)(c_j - off),
    at most (s / 2) D sum_j |c_j - off|.  Checked in float64 on random,
    spiky and adversarial cases (one dominant query element, every other
    element's rounding error of one sign, codes far from their offset):
    always below 5 % of the float32 tolerance 1e-5 ||q|| ||x^||."""
    g = np.random.default_rng(3)
    worst = 0.0
    for d in (24, 96, 768, 4096):
        for trial in range(40):
            kind = trial % 4
            if kind == 0:
                q = g.standard_normal(d)
            elif kind == 1:
                q = g.standard_normal(d) * (g.random(d) < 0.02) + 1e-3 * g.standard_normal(d)
            elif kind == 2:
                q = np.full(d, 1.0) + 1e-6 * g.standard_normal(d)
            else:
                q = np.full(d, 0.3e-7)     # rounding errors all of one sign
                q[0] = 1.0
            q = q.astype(np.float32).astype(np.float64)
            if kind == 3:
                c = np.zeros(d)
                c[0] = 15.0
            else:
                c = g.integers(0, 16, d).astype(np.float64)
            lo, step = g.standard_normal(), abs(g.standard_normal()) + 1e-3
            x = lo + step * c
            s = 2.0 ** (np.floor(np.log2(np.abs(q).max())) - 30)
            qq = np.rint(q / s)
            assert np.abs(qq).max() < 2 ** 31
            exact = q @ x
            approx = (lo + 8 * step) * q.sum() + step * s * (qq @ (c - 8))
            err = abs(approx - exact)
            bound = (s / 2) * step * np.abs(c - 8).sum() * (1 + 1e-9) + 1e-12 * abs(exact)
            assert err <= bound
            tol = 1e-5 * np.linalg.norm(q) * np.linalg.norm(x)
            worst = max(worst, err / tol)
    assert worst < 0.05

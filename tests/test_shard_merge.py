"""Row-sharded search (each rank one slot range of the database): the
per-shard top-k lists, all-gathered over gloo by two CPU ranks and merged,
equal the oracle's search over the whole database (first level), and the
oracle's re-rank of the union of the shards' candidates (two levels)."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
import synth
from paper_2402_02044_b300.shard import gather_merge, merge_topk

N, D, NQ, K, K1 = 3000, 48, 6, 10, 40


def _data(metric):
    mix = synth.Mixture(d=D, n_comp=8, sigma=0.3, normalize=metric == "ip", seed=77)
    x = mix.base(N)
    q = mix.queries(NQ)
    means = synth.sample_mean(x)[None]
    return x, q, means, O.encode(x, means, 4, 8)


def test_merge_orders_by_score_then_id_and_pads_last():
    ids = torch.tensor([[5, 3, -1, 9, 2]])
    sc = torch.tensor([[1.0, 1.0, float("inf"), 0.5, 2.0]])
    i, s = merge_topk(ids, sc, 4, "l2")
    assert i.tolist() == [[9, 3, 5, 2]] and s.tolist() == [[0.5, 1.0, 1.0, 2.0]]
    i, s = merge_topk(ids, torch.tensor([[1.0, 1.0, float("-inf"), 0.5, 2.0]]), 5, "ip")
    assert i.tolist() == [[2, 3, 5, 9, -1]] and s[0, -1].item() == float("-inf")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, metric, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x, q, means, enc = _data(metric)
    base = rank * N // world
    rows = np.arange(base, (rank + 1) * N // world)
    shard = O.take(enc, rows)
    res = {}
    for name, k1 in (("first", 0), ("two", K1)):
        ids, sc = O.search_exhaustive(shard, means, q, k1, K, metric)
        mi, ms = gather_merge(torch.from_numpy(ids), torch.from_numpy(sc), base, K, metric)
        res[name] = (mi.numpy(), ms.numpy())
    out[rank] = res
    dist.destroy_process_group()


def _run(metric):
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, metric, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    return dict(out), world


def _check(metric):
    out, world = _run(metric)
    x, q, means, enc = _data(metric)
    # first level: exactly the whole-database search
    gi, gs = O.search_exhaustive(enc, means, q, 0, K, metric)
    # two levels: the re-rank of the union of the shards' first-level candidates
    cands = []
    for r in range(world):
        base = r * N // world
        ci, _ = O.search_exhaustive(O.take(enc, np.arange(base, (r + 1) * N // world)), means, q, 0, K1, metric)
        cands.append(np.where(ci >= 0, ci + base, -1))
    ti, ts = O.rerank(enc, means, q, np.concatenate(cands, 1), K, metric)
    for r in range(world):
        fi, fs = out[r]["first"]
        assert np.array_equal(fi, gi) and np.array_equal(fs, gs)
        wi, ws = out[r]["two"]
        assert np.array_equal(wi, ti) and np.allclose(ws, ts, rtol=0, atol=0)


def test_sharded_search_over_gloo_l2():
    _check("l2")


def test_sharded_search_over_gloo_ip():
    _check("ip")

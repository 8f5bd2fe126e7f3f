"""The continuous-batching serving loop on the GPU: every request's result is
the same alone and mixed with others (uneven sizes, different k, several
lanes in flight, CUDA graphs or not), updates become visible at epoch
boundaries, and admission rejects what can never fit."""
import threading

import numpy as np
import pytest
import torch

import oracle as O
import synth
from helpers import lib_store

pytestmark = pytest.mark.gpu


def _setup(n=30000, d=128, metric="ip"):
    mix = synth.Mixture(d=d, n_comp=32, sigma=0.3, normalize=metric == "ip", seed=61)
    x = mix.base(n)
    means = synth.sample_mean(x)[None]
    st, _ = lib_store(x, means, 4, 8, metric, capacity=n + 5000)
    return mix, x, means, st


@pytest.mark.parametrize("graphs", [False, True])
def test_results_alone_equal_results_in_the_mix(graphs):
    from paper_2402_02044_b300.serve import Server
    mix, x, means, st = _setup()
    g = np.random.default_rng(0)
    sizes = [1, 7, 64, 3, 200, 33, 1, 512, 18, 90]
    ks = [10, 100, 10, 50, 10, 100, 1, 10, 20, 100]
    qs = [mix.rows(1000 * i, 1000 * i + n, stream=11) for i, n in enumerate(sizes)]
    srv = Server(st, lanes=3, max_batch=1024, k1=100, kmax=100, precision="fp16", use_graphs=graphs)
    alone = []
    for q, k in zip(qs, ks):
        alone.append(srv.submit_query(q, k).result(timeout=60))
    # mixed: all at once from several client threads
    futs = [None] * len(qs)

    def client(idx):
        for i in idx:
            futs[i] = srv.submit_query(qs[i], ks[i])
    threads = [threading.Thread(target=client, args=(list(range(j, len(qs), 3)),)) for j in range(3)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    mixed = [f.result(timeout=60) for f in futs]
    for (ai, asc, _), (mi, msc, _) in zip(alone, mixed):
        assert np.array_equal(ai, mi) and np.array_equal(asc, msc)
    # and the same as a direct search through the library
    for q, k, (ai, asc, _) in zip(qs, ks, alone):
        di, ds = st.search(torch.from_numpy(q).cuda(), k, 100, "fp16")
        assert np.array_equal(di.cpu().numpy(), ai) and np.array_equal(ds.cpu().numpy(), asc)
    s = srv.stats_summary()
    assert s["requests"] == 2 * len(qs) and s["p99_ms"] >= s["p50_ms"] > 0
    srv.close()
    st.close()


def test_requests_larger_than_a_batch_are_split_within_one_epoch():
    """A request of more rows than max_batch runs as parts of at most
    max_batch rows; its result equals the direct search, and updates
    submitted while it runs apply to all of its parts or to none."""
    from paper_2402_02044_b300.serve import Server
    mix, x, means, st = _setup(n=20000)
    srv = Server(st, lanes=2, max_batch=64, k1=50, kmax=10, precision="fp16")
    qs = [mix.rows(2000 * i, 2000 * i + n, stream=21) for i, n in enumerate([1, 200, 65, 130, 7])]
    res = [srv.submit_query(q, 10).result(timeout=60) for q in qs]
    for q, (ri, rs, _) in zip(qs, res):
        assert ri.shape == (len(q), 10)
        di, ds = st.search(torch.from_numpy(q).cuda(), 10, 50, "fp16")
        assert np.array_equal(di.cpu().numpy(), ri) and np.array_equal(ds.cpu().numpy(), rs)
    # a 400-row request (7 parts) with a delete of its current best answers behind it
    big = mix.rows(50000, 50400, stream=22)
    before = st.search(torch.from_numpy(big).cuda(), 10, 50, "fp16")[0].cpu().numpy()
    fq = srv.submit_query(big, 10)
    fd = srv.submit_delete(np.unique(before[:, 0]))
    gi, gs, ep = fq.result(timeout=60)
    fd.result(timeout=60)
    srv.drain()
    after = st.search(torch.from_numpy(big).cuda(), 10, 50, "fp16")[0].cpu().numpy()
    assert np.array_equal(gi, before) or np.array_equal(gi, after)
    srv.close()
    st.close()


def test_updates_become_visible_at_epoch_boundaries():
    from paper_2402_02044_b300.serve import Server
    mix, x, means, st = _setup(n=20000, d=64, metric="l2")
    srv = Server(st, lanes=2, max_batch=512, k1=50, kmax=10, precision="fp16")
    # the replay's live marks occupied slots: live ones and deleted ones
    # still held for older snapshots
    rep = O.SlotReplay(st.capacity)
    rep.insert(20000)
    rows = {i: x[i] for i in range(20000)}
    g = np.random.default_rng(5)
    held = np.zeros(0, np.int64)  # deleted at the previous boundary
    for step in range(3):
        live_now = rep.live.copy()
        live_now[held] = False
        dele = g.choice(np.nonzero(live_now)[0], 500, replace=False)
        new = mix.rows(100 * step, 100 * step + 700, stream=12)
        # the insert goes first: it is encoded when the scheduler stages it,
        # before the boundary that frees the slots held at the previous one
        # (a delete submitted first could reach a boundary of its own before
        # the insert is staged, and that boundary would free them earlier)
        fi = srv.submit_insert(new)
        fd = srv.submit_delete(dele)
        fq = srv.submit_query(new[:5], 10)          # queued behind the updates or before them
        ids_new = fi.result(timeout=60)
        assert fd.result(timeout=60) == 500
        # an epoch's inserts take the lowest slots neither live nor held; its
        # deletes are held until the next boundary, which frees the slots held
        # at this one
        ref_new = rep.insert(700)
        rep.delete(held)
        held = dele
        assert np.array_equal(np.sort(ids_new), np.sort(ref_new))
        for r, v in zip(ids_new, new):
            rows[int(r)] = v
        fq.result(timeout=60)
    srv.drain()
    live = rep.live.copy()
    live[held] = False
    assert st.stats() == live.sum()
    # the state after the last epoch: a fresh query equals the oracle
    live_ids = np.nonzero(live)[0]
    q = mix.queries(4)
    got_i, got_s, _ = srv.submit_query(q, 10).result(timeout=60)
    xs = np.zeros((st.capacity, 64), np.float32)
    for i in live_ids:
        xs[i] = rows[int(i)]
    enc = O.encode(xs, means, 4, 8)
    from helpers import TOL_FP16, check_two_level
    # the server runs the tensor-core first level (precision fp16); the same
    # scan on the store gives its first stage
    first = st.first_level(torch.from_numpy(q).cuda(), 50, "fp16")
    check_two_level(q, got_i, got_s, first, enc, means, "l2", 50, 10, TOL_FP16, live=live)
    srv.close()
    st.close()


def test_snapshot_views_and_held_deletes():
    """A view on a visibility snapshot keeps seeing the slots live when it was
    taken; lvq_delete_hold keeps deleted slots from reuse until lvq_release."""
    mix, x, means, st = _setup(n=3000, d=64)
    q = torch.from_numpy(mix.queries(4)).cuda()
    snap = st.live_snapshot()
    torch.cuda.synchronize()
    v = st.view()
    v.set_live(snap)
    bi, bs = v.search(q, 10, 50, "fp16")
    top = np.unique(bi[:, 0].cpu().numpy())
    assert int(st.delete_hold(torch.from_numpy(top).cuda()).item()) == len(top)
    vi, vs = v.search(q, 10, 50, "fp16")
    assert torch.equal(vi, bi) and torch.equal(vs, bs)
    si, _ = st.search(q, 10, 50, "fp16")
    assert not np.isin(si.cpu().numpy(), top).any()
    # held slots are skipped by inserts (the lowest free slots lie above 3000)
    add = torch.from_numpy(mix.rows(9000, 9000 + len(top), stream=31)).cuda()
    ids1 = st.insert(add).cpu().numpy()
    assert not np.isin(ids1, top).any()
    st.delete(torch.from_numpy(ids1).cuda())
    st.release(torch.from_numpy(top).cuda())
    ids2 = st.insert(add).cpu().numpy()
    assert np.array_equal(np.sort(ids2), np.sort(top))
    v.set_live(None)
    vi, vs = v.search(q, 10, 50, "fp16")
    si, ss = st.search(q, 10, 50, "fp16")
    assert torch.equal(vi, si) and torch.equal(vs, ss)
    v.close()
    st.close()


def test_admission_rejects_what_cannot_fit():
    from paper_2402_02044_b300.serve import Server
    mix, x, means, st = _setup(n=5000, d=32)
    srv = Server(st, lanes=1, max_batch=256, k1=50, kmax=10, hbm_budget=20000)
    with pytest.raises(MemoryError):
        srv.submit_query(mix.queries(200), 10).result(timeout=10)
    assert srv.submit_query(mix.queries(2), 10).result(timeout=30)[0].shape == (2, 10)
    assert srv.stats_summary()["rejected"] == 1
    srv.close()
    st.close()

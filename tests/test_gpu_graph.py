"""GPU parity of the greedy beam search over a graph (lvq_search_graph,
Alg. 1).

* Integer-valued data (every decoded vector and query an integer vector with
  small entries): the kernel's float32 first-level scores are then exact, so
  every decision of the search is the oracle's and the results must equal
  the oracle's beam search id for id and score for score, ties included
  (both order by (score, id)).
* Mixture data: every returned score is right; a query whose oracle search
  made no decision on two scores within the float32 tolerance must return
  exactly the oracle's ids; deleted nodes never appear, and the two-level
  search re-ranks the beam's own candidates."""
import numpy as np
import pytest
import torch

import oracle as O
from helpers import TOL_FP32, _check_boundary, check_no_device_error, check_scores, check_sorted, gmm_case, lib_store

pytestmark = pytest.mark.gpu


def _setup(metric, n=20000, d=64, nq=12, seed=41):
    from paper_2402_02044_b300.graph import knn_graph
    x, q, means = gmm_case(n, d, 32, metric, nq, seed=seed)
    st, _ = lib_store(x, means, 4, 8, metric)
    xt = torch.from_numpy(x).cuda()
    graph = knn_graph(st, xt, 24, 8, seed=seed)
    starts = np.random.default_rng(seed).choice(n, 16, replace=False).astype(np.int64)
    return x, q, means, st, graph, starts


def _integer_case(n, d, nq, seed):
    """Rows x = l + c with c in [0, 15] (both ends present, so the 4-bit step
    is exactly 1 and the codes are c), l a small integer, the centre zero;
    queries small integers.  Decoded vectors equal x, and float32 sums of
    their products and squared differences with the queries are exact."""
    g = np.random.default_rng(seed)
    c = g.integers(0, 16, (n, d))
    c[:, 0], c[:, 1] = 0, 15
    lower = g.integers(-8, 9, n)
    x = (lower[:, None] + c).astype(np.float32)
    q = g.integers(-8, 24, (nq, d)).astype(np.float32)
    return x, q, np.zeros((1, d), np.float32)


@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_graph_search_equals_the_oracle_on_exact_scores(metric):
    from paper_2402_02044_b300.graph import knn_graph
    n, d, nq = 6000, 64, 16
    x, q, means = _integer_case(n, d, nq, seed=7 if metric == "l2" else 8)
    st, _ = lib_store(x, means, 4, 8, metric)
    enc = O.encode(x, means, 4, 8)
    assert np.array_equal(O.decode_first(enc, means), x.astype(np.float64))
    graph = knn_graph(st, torch.from_numpy(x).cuda(), 12, 4, seed=3)
    starts = np.random.default_rng(5).choice(n, 8, replace=False).astype(np.int64)
    dead = np.arange(0, n, 17)
    st.delete(torch.from_numpy(dead).cuda())
    live = np.ones(n, bool)
    live[dead] = False
    qt = torch.from_numpy(q).cuda()
    for L, exp in ((32, 0), (64, 40), (16, 500)):
        gi, gs = st.search_graph(qt, graph, torch.from_numpy(starts).cuda(), 10, 0, L=L, max_expand=exp)
        oi, os_ = O.beam_search(enc, means, q, graph.cpu().numpy(), starts, L, 10, metric, live=live,
                                max_expand=exp if exp else 4 * L)
        assert np.array_equal(gi.cpu().numpy(), oi), (L, exp)
        assert np.array_equal(gs.cpu().numpy().astype(np.float64), os_), (L, exp)
    check_no_device_error(st)
    st.close()


@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_graph_search_matches_the_oracle(metric):
    x, q, means, st, graph, starts = _setup(metric)
    enc = O.encode(x, means, 4, 8)
    qt = torch.from_numpy(q).cuda()
    L, exp = 64, 256
    st_t = torch.from_numpy(starts).cuda()
    gi, gs = st.search_graph(qt, graph, st_t, 10, 0, L=L, max_expand=exp)
    check_sorted(gs, metric)
    check_scores(q, gi, gs, enc, means, metric, 1, TOL_FP32)
    # the oracle's whole final list (k = L) and its near-tie flags
    oi, _, amb = O.beam_search(enc, means, q, graph.cpu().numpy(), starts, L, L, metric, max_expand=exp,
                               tol=TOL_FP32)
    gi_np, gs_np = gi.cpu().numpy(), gs.cpu().numpy()
    xh = O.decode_first(enc, means)
    for i in np.nonzero(~amb)[0]:
        # no decision of the search rested on a near-tie: the listed nodes
        # are the oracle's, and the k best of them agree up to ties at k
        listed = np.unique(oi[i][oi[i] >= 0])
        s = O.score(q[i], xh[listed], metric)[0]
        scl = np.maximum(np.abs(s), np.linalg.norm(q[i].astype(np.float64)) * np.linalg.norm(xh[listed], axis=1))
        _check_boundary(i, listed, s, scl, gi_np[i], gs_np[i], metric, 10, TOL_FP32)
    # two levels: the beam's 40 best re-ranked to 10 by both levels
    ti, ts = st.search_graph(qt, graph, st_t, 10, 40, L=L, max_expand=exp)
    check_sorted(ts, metric)
    check_scores(q, ti, ts, enc, means, metric, 2, TOL_FP32)
    fi, fs = st.search_graph(qt, graph, st_t, 40, 0, L=L, max_expand=exp)
    ti_np, ts_np, fi_np = ti.cpu().numpy(), ts.cpu().numpy(), fi.cpu().numpy()
    x2 = O.decode_second(enc, means)
    for i in range(len(q)):
        pool = np.unique(fi_np[i][fi_np[i] >= 0])
        s = O.score(q[i], x2[pool], metric)[0]
        scl = np.maximum(np.abs(s), np.linalg.norm(q[i].astype(np.float64)) * np.linalg.norm(x2[pool], axis=1))
        _check_boundary(i, pool, s, scl, ti_np[i], ts_np[i], metric, 10, TOL_FP32)
    ei, _ = st.search(qt, 10, 40, "fp32")
    rec = np.mean([len(set(a) & set(b)) / 10 for a, b in zip(ti_np, ei.cpu().numpy())])
    assert rec >= 0.8, rec  # an approximate search on an approximate graph
    check_no_device_error(st)
    st.close()


def test_graph_search_skips_deleted_nodes_and_checks_arguments():
    from paper_2402_02044_b300 import lvq as L_
    x, q, means, st, graph, starts = _setup("l2", n=5000, nq=4, seed=43)
    dead = np.arange(0, 5000, 3)
    st.delete(torch.from_numpy(dead).cuda())
    qt = torch.from_numpy(q).cuda()
    gi, _ = st.search_graph(qt, graph, torch.from_numpy(starts).cuda(), 10, 20, L=32)
    assert not np.isin(gi.cpu().numpy(), dead).any()
    with pytest.raises(L_.LVQError):
        st.search_graph(qt, graph, torch.from_numpy(starts).cuda(), 10, 20, L=8)  # L < k1
    check_no_device_error(st)
    st.close()

"""GPU parity of the greedy beam search over a graph (lvq_search_graph,
Alg. 1): on a navigable graph built by the library (first-level k-NN plus
random long-range edges) the first-level results agree with the oracle's
beam search on the same graph, starts, L and expansion limit (up to the
rare step where float32 and float64 scores order two candidates
differently), every returned score is right, deleted nodes never appear,
and the two-level search finds most of the exhaustive search's neighbours."""
import numpy as np
import pytest
import torch

import oracle as O
from helpers import TOL_FP32, check_no_device_error, check_scores, check_sorted, gmm_case, lib_store

pytestmark = pytest.mark.gpu


def _setup(metric, n=20000, d=64, nq=12, seed=41):
    from paper_2402_02044_b300.graph import knn_graph
    x, q, means = gmm_case(n, d, 32, metric, nq, seed=seed)
    st, _ = lib_store(x, means, 4, 8, metric)
    xt = torch.from_numpy(x).cuda()
    graph = knn_graph(st, xt, 24, 8, seed=seed)
    starts = np.random.default_rng(seed).choice(n, 16, replace=False).astype(np.int64)
    return x, q, means, st, graph, starts


@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_graph_search_matches_the_oracle(metric):
    x, q, means, st, graph, starts = _setup(metric)
    enc = O.encode(x, means, 4, 8)
    qt = torch.from_numpy(q).cuda()
    L, exp = 64, 256
    gi, gs = st.search_graph(qt, graph, torch.from_numpy(starts).cuda(), 10, 0, L=L, max_expand=exp)
    check_sorted(gs, metric)
    check_scores(q, gi, gs, enc, means, metric, 1, TOL_FP32)
    oi, _ = O.beam_search(enc, means, q, graph.cpu().numpy(), starts, L, 10, metric, max_expand=exp)
    agree = np.mean([len(set(a) & set(b)) / 10 for a, b in zip(gi.cpu().numpy(), oi)])
    assert agree >= 0.95, agree
    # two levels: the beam's 40 best re-ranked to 10 find the exhaustive neighbours
    ti, ts = st.search_graph(qt, graph, torch.from_numpy(starts).cuda(), 10, 40, L=L, max_expand=exp)
    check_sorted(ts, metric)
    check_scores(q, ti, ts, enc, means, metric, 2, TOL_FP32)
    ei, _ = st.search(qt, 10, 40, "fp32")
    rec = np.mean([len(set(a) & set(b)) / 10 for a, b in zip(ti.cpu().numpy(), ei.cpu().numpy())])
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

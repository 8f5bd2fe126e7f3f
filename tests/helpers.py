"""Shared helpers of the GPU parity tests: build stores through the C ABI and
compare their results with the CPU oracle within the stated tolerances."""
import numpy as np
import torch

import oracle as O
import synth

TOL_FP32 = 1e-5    # relative, float32 scoring (scale: max(|s|, ||q|| ||x^||))
TOL_FP16 = 2e-3    # relative, float16 tensor-core first level


def _np(t):
    return t.cpu().numpy() if torch.is_tensor(t) else np.asarray(t)


def lib_store(x, means, bits1, bits2, metric, capacity=None, grid2="text"):
    from paper_2402_02044_b300 import Store, build
    build.build()
    st = Store(x.shape[1], bits1, bits2, means, metric, capacity or len(x), grid2=grid2)
    ids = st.insert(torch.from_numpy(np.ascontiguousarray(x)).cuda()) if len(x) else None
    return st, ids


def gmm_case(n, d, comps, metric, nq, seed, normalize=None, n_means=1):
    normalize = (metric == "ip") if normalize is None else normalize
    mix = synth.Mixture(d=d, n_comp=comps, sigma=0.3, normalize=normalize, seed=seed)
    x = mix.base(n)
    q = mix.queries(nq)
    if n_means == 1:
        means = synth.sample_mean(x)[None]
    else:
        means = synth.kmeans_means(x[: min(n, 20000)], n_means, seed=seed, iters=10)
    return x, q, means


def scale(q, xhat, metric):
    """Tolerance scale per (query, row): max(|s|, ||q|| ||x^||)."""
    qn = np.linalg.norm(np.atleast_2d(q).astype(np.float64), axis=1)[:, None]
    xn = np.linalg.norm(xhat, axis=1)[None, :]
    return qn * xn


def check_scores(q, ids, scores, enc, means, metric, level, tol):
    """Every returned (id, score) pair matches the oracle's score of that id."""
    ids, scores = _np(ids), _np(scores)
    for i in range(len(q)):
        sel = ids[i] >= 0
        if not sel.any():
            continue
        rows = ids[i][sel]
        xh = O.decode(O.take(enc, rows), means, level)
        ref = O.score(q[i], xh, metric)[0]
        sc = np.maximum(np.abs(ref), scale(q[i], xh, metric)[0])
        err = np.abs(scores[i][sel].astype(np.float64) - ref)
        assert np.all(err <= tol * sc), (i, float((err / sc).max()))


def check_sorted(scores, metric):
    s = scores.cpu().numpy() if torch.is_tensor(scores) else scores
    d = np.diff(s, axis=1)
    d = d[np.isfinite(d)]
    assert np.all(d >= 0) if metric == "l2" else np.all(d <= 0)


def _scale_of(q_i, xh_rows, s_ref):
    """max(|s|, ||q|| ||x^||) per row: the tolerance scale of reading (xi)."""
    qn = float(np.linalg.norm(np.asarray(q_i, dtype=np.float64)))
    return np.maximum(np.abs(s_ref), qn * np.linalg.norm(xh_rows, axis=1))


def _check_boundary(i, pool, s_ref, scale_, got_ids, got_scores, metric, k, tol):
    """One query's k best over ``pool``: the GPU's ids (best first) against the
    oracle's, at the stated tolerance.

    The GPU ranks by its own scores s', each within tol * scale of the
    oracle's s (check_scores verifies that for every returned id).  So an id
    the oracle ranks in and the GPU leaves out must have s within
    tol * scale of the GPU's own k-th returned score s'_k (on the better
    side), and an id the GPU returns but the oracle does not must have s
    within tol * scale of s'_k on the worse side; every other id must agree.
    """
    order = O.best_first(s_ref, pool, metric)
    n_exp = min(k, len(pool))
    ref = pool[order[:n_exp]]
    valid = got_ids >= 0
    got = got_ids[valid]
    assert len(got) == n_exp, (i, len(got), n_exp)
    assert np.all(valid[:n_exp]), i
    assert len(set(got.tolist())) == len(got), i
    pos = {int(v): j for j, v in enumerate(pool)}
    assert all(int(g) in pos for g in got), (i, "an id outside the searched set")
    if n_exp == 0:
        return
    gk = float(got_scores[n_exp - 1])
    sign = 1.0 if metric == O.L2 else -1.0
    for h in set(ref.tolist()) - set(got.tolist()):
        j = pos[h]
        # left out by the GPU: s'(h) is no better than s'_k, and |s' - s| <= tol * scale
        assert sign * (s_ref[j] - gk) >= -tol * scale_[j], (i, "missed", h, s_ref[j], gk)
    for g in set(got.tolist()) - set(ref.tolist()):
        j = pos[g]
        assert sign * (s_ref[j] - gk) <= tol * scale_[j], (i, "extra", g, s_ref[j], gk)


def _pool(i, n, live, cand_ids):
    pool = np.nonzero(live)[0] if cand_ids is None else np.unique(
        cand_ids[i][(cand_ids[i] >= 0) & (cand_ids[i] < n)])
    return pool[live[pool]].astype(np.int64)


def check_topk_ids(q, gpu_ids, gpu_scores, enc, means, metric, k, tol, live=None, level=1, cand_ids=None):
    """A single-stage top-k (the k best live rows, or candidates, by the
    score at ``level``): returned scores within ``tol`` of the oracle's and
    ids equal to the oracle's up to ties at the k boundary within ``tol``
    (``_check_boundary``)."""
    gpu_ids = _np(gpu_ids)
    gpu_scores = _np(gpu_scores)
    check_scores(q, gpu_ids, gpu_scores, enc, means, metric, level, tol)
    n = len(enc["lower"])
    live = np.ones(n, bool) if live is None else live
    for i in range(len(q)):
        pool = _pool(i, n, live, cand_ids)
        xh = O.decode(O.take(enc, pool), means, level)
        s = O.score(q[i], xh, metric)[0]
        _check_boundary(i, pool, s, _scale_of(q[i], xh, s), gpu_ids[i], gpu_scores[i], metric, k, tol)


def check_two_level(q, gpu_ids, gpu_scores, first, enc, means, metric, k1, k, tol1, live=None, cand_ids=None):
    """Two-stage search (first level k1 best, re-ranked by both levels to k).

    ``first`` = (ids, scores) of the GPU's first stage alone for the same
    queries (lvq_search_first_level, or the candidate search with k1 = 0 and
    k = k1): the same scan gives the same k1 set.  Stage 1 is held to the
    first-level tolerance ``tol1`` against the oracle's k1 best; stage 2 must
    be the oracle's two-level re-rank of the GPU's own k1 set, at the float32
    tolerance of the re-rank (both with ``_check_boundary``)."""
    gpu_ids, gpu_scores = _np(gpu_ids), _np(gpu_scores)
    fi, fs = _np(first[0]), _np(first[1])
    check_topk_ids(q, fi, fs, enc, means, metric, k1, tol1, live=live, level=1, cand_ids=cand_ids)
    check_scores(q, gpu_ids, gpu_scores, enc, means, metric, 2, TOL_FP32)
    for i in range(len(q)):
        pool = np.unique(fi[i][fi[i] >= 0]).astype(np.int64)
        xh = O.decode(O.take(enc, pool), means, 2)
        s = O.score(q[i], xh, metric)[0]
        _check_boundary(i, pool, s, _scale_of(q[i], xh, s), gpu_ids[i], gpu_scores[i], metric, k, TOL_FP32)


def check_rerank(q, gpu_ids, gpu_scores, enc, means, metric, cand, k, live=None):
    """lvq_rerank: each query's live, distinct, in-range candidates ordered by
    the two-level score, the k best, at the float32 tolerance."""
    check_topk_ids(q, gpu_ids, gpu_scores, enc, means, metric, k, TOL_FP32, live=live, level=2, cand_ids=cand)


def check_no_device_error(st):
    """No bounded device wait expired and no other sticky error was recorded."""
    from paper_2402_02044_b300 import lvq as L
    code, msg = L.lvq_last_error(st.handle)
    assert code == 0, msg

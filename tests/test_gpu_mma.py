"""GPU parity of the tcgen05 tensor-core first level (LVQ_FP16_MMA).

The queries are rounded to float16 and the products accumulate in float32:
scores must match the float64 oracle within 2e-3 relative to
max(|s|, ||q|| ||x^||), ids up to near-ties within that tolerance.  The
cases cover every query-tile width (16, 32, 64, 128), ragged query counts
(one tile partly filled), ragged dimensionalities, both code widths, both
metrics, several centring means and a database that is not a whole number
of 128-row tiles.
"""
import numpy as np
import pytest
import torch

import oracle as O
from helpers import (TOL_FP16, TOL_FP32, check_no_device_error, check_scores, check_sorted, check_topk_ids,
                     check_two_level, gmm_case, lib_store)

pytestmark = pytest.mark.gpu

CASES = [
    # n, d, comps, metric, bits1, bits2, n_means, nq, k1, k
    (5000, 768, 32, "ip", 4, 8, 1, 1, 100, 10),
    (5000, 768, 32, "ip", 4, 8, 1, 5, 100, 10),
    (7777, 768, 64, "ip", 4, 8, 16, 33, 100, 10),
    (6000, 768, 32, "ip", 4, 8, 1, 64, 100, 10),
    (9000, 768, 32, "ip", 4, 8, 1, 130, 100, 10),
    (6000, 96, 16, "l2", 4, 8, 1, 40, 50, 10),
    (4099, 100, 8, "l2", 4, 8, 1, 17, 64, 7),
    (3000, 200, 32, "l2", 4, 8, 16, 20, 40, 10),
    (5000, 96, 32, "l2", 8, 8, 1, 24, 30, 10),
    (3000, 768, 16, "ip", 8, 8, 4, 9, 100, 10),
    (4000, 768, 32, "ip", 8, 0, 1, 40, 0, 10),     # LVQ-8 single level at d = 768
    (4000, 768, 32, "l2", 4, 0, 4, 20, 0, 10),     # LVQ-4 single level, M-LVQ
    (2000, 4096, 8, "ip", 4, 8, 1, 20, 64, 10),    # the largest d (narrow query tiles)
    (3000, 64, 16, "l2", 4, 8, 256, 40, 40, 10),   # the most centres
    (6000, 128, 16, "ip", 4, 8, 1, 50, 512, 10),   # the largest k1
]


def _id(c):
    return "n%d-d%d-%s-%dx%d-M%d-q%d" % (c[0], c[1], c[3], c[4], c[5], c[6], c[7])


@pytest.mark.parametrize("case", CASES, ids=_id)
def test_tensor_core_first_level_and_search(case):
    n, d, comps, metric, b1, b2, m, nq, k1, k = case
    x, q, means = gmm_case(n, d, comps, metric, nq, seed=300 + d + nq, n_means=m)
    st, ids = lib_store(x, means, b1, b2, metric)
    mid = st.export(ids)["mean_id"].cpu().numpy()
    enc = O.encode(x, means, b1, b2, mean_id=mid)
    qt = torch.from_numpy(q).cuda()
    kk = k1 if k1 else k
    fi, fs = st.first_level(qt, kk, "fp16")
    check_sorted(fs, metric)
    check_scores(q, fi, fs, enc, means, metric, 1, TOL_FP16)
    check_topk_ids(q, fi, fs, enc, means, metric, kk, TOL_FP16, level=1)
    gi, gs = st.search(qt, k, k1, "fp16")
    check_sorted(gs, metric)
    if b2 and k1:
        # re-rank distances are float32
        check_scores(q, gi, gs, enc, means, metric, 2, TOL_FP32)
        check_two_level(q, gi, gs, (fi, fs), enc, means, metric, k1, k, TOL_FP16)
    else:
        check_scores(q, gi, gs, enc, means, metric, 1, TOL_FP16)
        check_topk_ids(q, gi, gs, enc, means, metric, k, TOL_FP16, level=1)
    check_no_device_error(st)
    st.close()


@pytest.mark.parametrize("mma_n", [16, 32, 64, 128])
def test_every_tile_width_gives_the_same_candidates(mma_n):
    x, q, means = gmm_case(4000, 768, 32, "ip", 70, seed=77)
    st, ids = lib_store(x, means, 4, 8, "ip")
    enc = O.encode(x, means, 4, 8)
    qt = torch.from_numpy(q).cuda()
    st.set_tuning(mma_n=mma_n)
    fi, fs = st.first_level(qt, 64, "fp16")
    check_scores(q, fi, fs, enc, means, "ip", 1, TOL_FP16)
    check_topk_ids(q, fi, fs, enc, means, "ip", 64, TOL_FP16, level=1)
    # fewer CTAs than SMs: longer segments, same results
    st.set_tuning(mma_n=mma_n, mma_ctas=7)
    fi2, fs2 = st.first_level(qt, 64, "fp16")
    assert torch.equal(fi, fi2) and torch.equal(fs, fs2)
    check_no_device_error(st)
    st.close()


def test_tensor_core_respects_deletes_and_padding():
    x, q, means = gmm_case(3000, 128, 8, "l2", 12, seed=8)
    st, ids = lib_store(x, means, 4, 8, "l2")
    g = np.random.default_rng(2)
    dead = np.unique(g.integers(0, 3000, 2000))
    st.delete(torch.from_numpy(dead).cuda())
    live = np.ones(3000, bool)
    live[dead] = False
    enc = O.encode(x, means, 4, 8)
    qt = torch.from_numpy(q).cuda()
    gi, gs = st.search(qt, 10, 40, "fp16")
    assert not np.isin(gi.cpu().numpy(), dead).any()
    check_two_level(q, gi, gs, st.first_level(qt, 40, "fp16"), enc, means, "l2", 40, 10, TOL_FP16, live=live)
    keep = np.nonzero(live)[0][:2]
    st.delete(torch.from_numpy(np.nonzero(live)[0][2:]).cuda())
    gi, gs = st.search(qt, 10, 40, "fp16")
    gi = gi.cpu().numpy()
    assert np.all(np.sort(gi[:, :2], axis=1) == keep) and np.all(gi[:, 2:] == -1)
    check_no_device_error(st)
    st.close()


def test_fp16_and_fp32_paths_both_match_the_oracle():
    """The float16 tensor-core and the float32 first levels each give the
    oracle's two-level search, element by element at their own tolerances,
    and their recall@10 against the oracle's exact top-10 over the decoded
    vectors is the oracle's own."""
    x, q, means = gmm_case(20000, 768, 64, "ip", 48, seed=12)
    st, ids = lib_store(x, means, 4, 8, "ip")
    enc = O.encode(x, means, 4, 8)
    qt = torch.from_numpy(q).cuda()
    truth, _ = O.ground_truth(enc, means, q, 10, "ip")
    ref_i, _ = O.search_exhaustive(enc, means, q, 100, 10, "ip")
    for prec, tol in (("fp16", TOL_FP16), ("fp32", TOL_FP32)):
        gi, gs = st.search(qt, 10, 100, prec)
        check_two_level(q, gi, gs, st.first_level(qt, 100, prec), enc, means, "ip", 100, 10, tol)
        assert abs(O.recall_at_k(gi.cpu().numpy(), truth, 10) - O.recall_at_k(ref_i, truth, 10)) <= 0.01, prec
    check_no_device_error(st)
    st.close()


@pytest.mark.parametrize("k1", [200, 512])
def test_large_k1_with_full_candidate_buffers(k1):
    """k1 above 128 gives per-(CTA, query) candidate buffers of 1024 keys;
    with few CTAs each scans thousands of rows, so the buffers fill and are
    cut many times: no candidate may be lost in a cut (every first-level
    and two-level result equals the oracle's)."""
    x, q, means = gmm_case(30000, 96, 16, "l2", 24, seed=131 + k1)
    st, ids = lib_store(x, means, 4, 8, "l2")
    enc = O.encode(x, means, 4, 8)
    qt = torch.from_numpy(q).cuda()
    for ctas in (7, 0):
        st.set_tuning(mma_ctas=ctas)
        fi, fs = st.first_level(qt, k1, "fp16")
        check_topk_ids(q, fi, fs, enc, means, "l2", k1, TOL_FP16, level=1)
        gi, gs = st.search(qt, 10, k1, "fp16")
        check_two_level(q, gi, gs, (fi, fs), enc, means, "l2", k1, 10, TOL_FP16)
    check_no_device_error(st)
    st.close()

"""GPU parity of the small-batch integer first level (LVQ_INT16).

Each query is rounded to 16-bit integers with one scale per query
(max|q| / 32767) and its products with the codes are exact in integers, so
the only error is the rounding of q: at most max|q| / 65534 per element,
below float16's relative error for every element larger than max|q| / 32.
Scores must match the float64 oracle within the float16 tolerance (2e-3
relative to max(|s|, ||q|| ||x^||)), ids up to near-ties within it.  The
cases cover 1 to 4 queries (one, two and four query slots), both code widths,
both metrics, several centring means, ragged dimensionalities, a database of
many tiles per CTA (candidate buffers cut back many times), a code row longer
than a TMA ring (8-bit, d = 768), and k1 up to its limit (512).
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
    (5000, 768, 32, "ip", 4, 8, 16, 3, 100, 10),
    (150000, 96, 32, "l2", 4, 8, 1, 2, 100, 10),
    (150000, 96, 32, "ip", 4, 8, 4, 4, 50, 10),
    (6000, 96, 16, "l2", 4, 8, 1, 2, 50, 10),
    (4099, 100, 8, "l2", 4, 8, 1, 3, 64, 7),
    (5000, 96, 32, "l2", 8, 8, 1, 4, 30, 10),
    (3000, 768, 16, "ip", 8, 8, 4, 1, 100, 10),
    (30000, 200, 16, "l2", 4, 8, 1, 2, 512, 10),
    (100, 96, 4, "l2", 4, 8, 1, 4, 100, 10),
    (4000, 768, 32, "ip", 8, 0, 1, 2, 0, 10),      # LVQ-8 single level at d = 768
    (4000, 768, 32, "l2", 4, 0, 4, 3, 0, 10),      # LVQ-4 single level, M-LVQ
    (2000, 4096, 8, "l2", 4, 8, 1, 2, 64, 10),     # the largest d
    (3000, 64, 16, "ip", 4, 8, 256, 4, 40, 10),    # the most centres
]


def _id(c):
    return "n%d-d%d-%s-%dx%d-M%d-q%d-k%d" % (c[0], c[1], c[3], c[4], c[5], c[6], c[7], c[8])


@pytest.mark.parametrize("case", CASES, ids=_id)
def test_integer_first_level_and_search(case):
    n, d, comps, metric, b1, b2, m, nq, k1, k = case
    x, q, means = gmm_case(n, d, comps, metric, nq, seed=500 + d + nq, n_means=m)
    st, ids = lib_store(x, means, b1, b2, metric)
    mid = st.export(ids)["mean_id"].cpu().numpy()
    enc = O.encode(x, means, b1, b2, mean_id=mid)
    qt = torch.from_numpy(q).cuda()
    k1_ = k1 if k1 else k
    kk = min(k1_, n)
    fi, fs = st.first_level(qt, k1_, "int16")
    check_sorted(fs, metric)
    check_scores(q, fi[:, :kk], fs[:, :kk], enc, means, metric, 1, TOL_FP16)
    check_topk_ids(q, fi[:, :kk], fs[:, :kk], enc, means, metric, kk, TOL_FP16, level=1)
    gi, gs = st.search(qt, k, k1, "int16")
    check_sorted(gs, metric)
    if b2 and k1:
        check_scores(q, gi, gs, enc, means, metric, 2, TOL_FP32)
        check_two_level(q, gi, gs, (fi, fs), enc, means, metric, k1, k, TOL_FP16)
    else:
        check_scores(q, gi, gs, enc, means, metric, 1, TOL_FP16)
        check_topk_ids(q, gi, gs, enc, means, metric, k, TOL_FP16, level=1)
    check_no_device_error(st)
    st.close()


def test_auto_takes_the_integer_scan_for_small_batches():
    from paper_2402_02044_b300 import lvq as L
    x, q, means = gmm_case(20000, 768, 32, "ip", 6, seed=91)
    st, ids = lib_store(x, means, 4, 8, "ip")
    qt = torch.from_numpy(q).cuda()
    L.lvq_profile_enable(st.handle, True)
    L.lvq_profile_read(st.handle)
    a_i, a_s = st.first_level(qt[:4], 100, "auto")
    prof = L.lvq_profile_read(st.handle)
    assert prof["scan_small"][1] == 1 and prof["scan_mma"][1] == 0
    b_i, b_s = st.first_level(qt[:4], 100, "int16")
    assert torch.equal(a_i, b_i) and torch.equal(a_s, b_s)
    L.lvq_profile_read(st.handle)
    st.first_level(qt[:5], 100, "auto")
    prof = L.lvq_profile_read(st.handle)
    assert prof["scan_small"][1] == 0 and prof["scan_mma"][1] == 1
    L.lvq_profile_enable(st.handle, False)
    with pytest.raises(L.LVQError):
        st.first_level(qt[:5], 100, "int16")
    # the integer and float32 first levels each give the oracle's two-level
    # search, element by element at their own tolerances
    enc = O.encode(x, means, 4, 8)
    for prec, tol in (("fp32", TOL_FP32), ("int16", TOL_FP16)):
        gi, gs = st.search(qt[:4], 10, 100, prec)
        check_two_level(q[:4], gi, gs, st.first_level(qt[:4], 100, prec), enc, means, "ip", 100, 10, tol)
    check_no_device_error(st)
    st.close()


def test_integer_scan_respects_deletes_and_zero_queries():
    x, q, means = gmm_case(3000, 128, 8, "l2", 3, seed=18)
    st, ids = lib_store(x, means, 4, 8, "l2")
    g = np.random.default_rng(4)
    dead = np.unique(g.integers(0, 3000, 2000))
    st.delete(torch.from_numpy(dead).cuda())
    live = np.ones(3000, bool)
    live[dead] = False
    enc = O.encode(x, means, 4, 8)
    q[1] = 0.0  # a zero query: every first-level score is <0, x^> terms only
    qt = torch.from_numpy(q).cuda()
    gi, gs = st.search(qt, 10, 40, "int16")
    assert not np.isin(gi.cpu().numpy(), dead).any()
    check_two_level(q, gi, gs, st.first_level(qt, 40, "int16"), enc, means, "l2", 40, 10, TOL_FP16, live=live)
    keep = np.nonzero(live)[0][:2]
    st.delete(torch.from_numpy(np.nonzero(live)[0][2:]).cuda())
    gi, gs = st.search(qt, 10, 40, "int16")
    gi = gi.cpu().numpy()
    assert np.all(np.sort(gi[:, :2], axis=1) == keep) and np.all(gi[:, 2:] == -1)
    check_no_device_error(st)
    st.close()

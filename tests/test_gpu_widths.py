"""GPU parity of the other code widths (Sec. 3.3: first levels of B1 = 2 ..
8 bits, residual levels of B2 = 2 .. 8 bits) and of the App. C listing's
signed residual grid: codes, bounds and steps bit-exact against the oracle
(both the plain encode and the stored records), and the searches (float32,
float16 tensor-core and integer first levels, the ID-gather form, caller-
given re-ranking, the graph search) equal to the oracle's element by element
at their tolerances."""
import numpy as np
import pytest
import torch

import oracle as O
from helpers import (TOL_FP16, TOL_FP32, check_no_device_error, check_rerank, check_scores, check_topk_ids,
                     check_two_level, gmm_case, lib_store)

pytestmark = pytest.mark.gpu

ENCODE_CASES = [
    # bits1, bits2, grid2, d, n_means
    (2, 8, "text", 96, 1), (3, 8, "text", 100, 4), (5, 8, "text", 64, 1), (6, 4, "text", 200, 1),
    (7, 2, "text", 33, 16), (8, 2, "text", 768, 1), (3, 2, "listing", 96, 1), (4, 8, "listing", 128, 4),
    (8, 2, "listing", 200, 1), (4, 0, "text", 96, 1), (6, 0, "text", 96, 1), (2, 3, "text", 768, 1),
]


def _eid(c):
    return "B%dx%d-%s-d%d-M%d" % c


@pytest.mark.parametrize("case", ENCODE_CASES, ids=_eid)
def test_encode_is_bit_exact_for_every_width_and_grid(case):
    b1, b2, grid2, d, m = case
    x, _, means = gmm_case(3000, d, 16, "l2", 1, seed=800 + b1 * 10 + b2, n_means=m)
    x[5] = 0.0                          # a constant vector (step 0)
    x[6, :] = np.linspace(-1, 1, d)     # an evenly spread row
    st, ids = lib_store(x, means, b1, b2, "l2", grid2=grid2)
    got = st.encode(torch.from_numpy(x).cuda())
    mid = got["mean_id"].cpu().numpy()
    if m > 1:
        # reading (vii): the GPU's centre is the nearest up to rounding
        ref_mid = O.assign_means(x, means)
        dd = ((x[:, None, :].astype(np.float64) - means[None].astype(np.float64)) ** 2).sum(-1)
        gap = dd[np.arange(len(x)), mid] - dd[np.arange(len(x)), ref_mid]
        assert np.all(gap <= 1e-5 * (x.astype(np.float64) ** 2).sum(1) + 1e-12)
    enc = O.encode(x, means, b1, b2, mean_id=mid, grid2=grid2)
    assert np.array_equal(got["codes1"].cpu().numpy(), enc["codes1"])
    assert np.array_equal(got["lower"].cpu().numpy().view(np.uint32), enc["lower"].view(np.uint32))
    assert np.array_equal(got["step"].cpu().numpy().view(np.uint32), enc["step"].view(np.uint32))
    if b2:
        c2 = got["codes2"].cpu().numpy()
        assert np.array_equal(c2.view(np.int8) if grid2 == "listing" else c2, enc["codes2"])
    # the stored records read back
    ex = st.export(ids)
    assert np.array_equal(ex["codes1"].cpu().numpy(), enc["codes1"])
    if b2:
        c2 = ex["codes2"].cpu().numpy()
        assert np.array_equal(c2.view(np.int8) if grid2 == "listing" else c2, enc["codes2"])
    check_no_device_error(st)
    st.close()


SEARCH_CASES = [
    # n, d, metric, bits1, bits2, grid2, n_means, nq, k1, k
    (6000, 96, "l2", 3, 8, "text", 1, 12, 50, 10),
    (5000, 200, "ip", 8, 2, "text", 4, 12, 40, 10),
    (6000, 96, "l2", 4, 8, "listing", 1, 12, 50, 10),
    (4000, 64, "ip", 2, 4, "text", 1, 12, 64, 10),
    (4000, 100, "l2", 6, 3, "listing", 1, 12, 40, 7),
]


def _sid(c):
    return "n%d-d%d-%s-B%dx%d-%s-M%d" % c[:7]


@pytest.mark.parametrize("case", SEARCH_CASES, ids=_sid)
def test_searches_for_every_width_and_grid(case):
    n, d, metric, b1, b2, grid2, m, nq, k1, k = case
    x, q, means = gmm_case(n, d, 16, metric, nq, seed=900 + b1 * 10 + b2, n_means=m)
    st, ids = lib_store(x, means, b1, b2, metric, grid2=grid2)
    mid = st.export(ids)["mean_id"].cpu().numpy()
    enc = O.encode(x, means, b1, b2, mean_id=mid, grid2=grid2)
    qt = torch.from_numpy(q).cuda()
    for prec, tol in (("fp32", TOL_FP32), ("fp16", TOL_FP16)):
        gi, gs = st.search(qt, k, k1, prec)
        check_two_level(q, gi, gs, st.first_level(qt, k1, prec), enc, means, metric, k1, k, tol)
    # the integer first level takes up to 4 queries per call
    gi, gs = st.search(qt[:4], k, k1, "int16")
    check_two_level(q[:4], gi, gs, st.first_level(qt[:4], k1, "int16"), enc, means, metric, k1, k, TOL_FP16)
    # ID-gather form and caller-given re-ranking
    g = np.random.default_rng(d)
    cand = g.integers(0, n, (nq, 600)).astype(np.int64)
    ct = torch.from_numpy(cand).cuda()
    gi, gs = st.search_candidates(qt, ct, k, k1)
    check_two_level(q, gi, gs, st.search_candidates(qt, ct, k1, 0), enc, means, metric, k1, k, TOL_FP32,
                    cand_ids=cand)
    ri, rs = st.rerank(qt, ct[:, :100].contiguous(), k)
    check_rerank(q, ri, rs, enc, means, metric, cand[:, :100], k)
    check_no_device_error(st)
    st.close()


def test_update_mean_with_the_listing_grid_and_three_bits():
    """The M-LVQ centre update re-encodes from the float32 two-level
    reconstruction on the listing's signed grid too, bit-exactly."""
    x, q, means = gmm_case(3000, 64, 8, "l2", 4, seed=91, n_means=2)
    st, ids = lib_store(x, means, 3, 5, "l2", grid2="listing")
    rec = st.export(ids)
    before = {k_: (v.cpu().numpy() if v is not None else None) for k_, v in rec.items()}
    if before["codes2"] is not None:
        before["codes2"] = before["codes2"].view(np.int8)
    enc = dict(before, bits1=3, bits2=5, grid2="listing")
    m = int(np.bincount(before["mean_id"], minlength=2).argmax())
    new_mu = (means[m] + np.float32(0.05)).astype(np.float32)
    cnt = st.update_mean(m, torch.from_numpy(new_mu).cuda())
    ref, means2, ref_cnt = O.update_mean(enc, means, m, new_mu)
    assert cnt == ref_cnt > 0
    after = st.export(ids)
    assert np.array_equal(after["codes1"].cpu().numpy(), ref["codes1"])
    assert np.array_equal(after["codes2"].cpu().numpy().view(np.int8), ref["codes2"])
    assert np.array_equal(after["lower"].cpu().numpy(), ref["lower"])
    assert np.array_equal(after["step"].cpu().numpy(), ref["step"])
    qt = torch.from_numpy(q).cuda()
    gi, gs = st.search(qt, 10, 40, "fp32")
    check_two_level(q, gi, gs, st.first_level(qt, 40, "fp32"), ref, means2, "l2", 40, 10, TOL_FP32)
    check_no_device_error(st)
    st.close()

"""GPU parity: every entry point of the C ABI against the CPU oracle.

Sizes are small enough for the oracle to finish in seconds yet span several
scan tiles (128 / 256 rows) with a ragged tail, ragged dimensionalities
(d = 100, 13), both bit widths, both metrics and several centring means.
Encoding is compared bit for bit; scores within 1e-5 (float32 path) of the
float64 oracle, relative to max(|s|, ||q|| ||x^||); ids exactly, up to
near-ties within that tolerance.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from helpers import (TOL_FP32, check_no_device_error, check_rerank, check_scores, check_sorted, check_topk_ids,
                     check_two_level, gmm_case, lib_store)

pytestmark = pytest.mark.gpu

ENC_CASES = [
    # n, d, comps, metric, bits1, bits2, n_means
    (3000, 96, 16, "l2", 8, 0, 1),
    (3000, 96, 16, "l2", 4, 8, 1),
    (2500, 768, 32, "ip", 4, 8, 1),
    (2000, 100, 8, "l2", 4, 8, 1),
    (777, 13, 4, "ip", 8, 8, 1),
    (4000, 200, 32, "l2", 4, 8, 16),
    (3000, 768, 64, "ip", 4, 8, 16),
]


def _enc_id(c):
    return "n%d-d%d-%s-%dx%d-M%d" % (c[0], c[1], c[3], c[4], c[5], c[6])


@pytest.mark.parametrize("case", ENC_CASES, ids=_enc_id)
def test_encode_is_bit_exact(case):
    n, d, comps, metric, b1, b2, m = case
    x, _, means = gmm_case(n, d, comps, metric, 1, seed=100 + d, n_means=m)
    st, ids = lib_store(x, means, b1, b2, metric)
    assert ids.cpu().tolist() == list(range(n))
    xt = torch.from_numpy(x).cuda()
    plain = st.encode(xt)
    stored = st.export(ids)
    for got in (plain, stored):
        mid = got["mean_id"].cpu().numpy()
        if m > 1:
            # near-ties may pick another centre; it must be (almost) nearest
            ref_mid = O.assign_means(x, means)
            x64, mu64 = x.astype(np.float64), means.astype(np.float64)
            d_got = ((x64 - mu64[mid]) ** 2).sum(1)
            d_ref = ((x64 - mu64[ref_mid]) ** 2).sum(1)
            assert np.all(d_got - d_ref <= 1e-5 * (x64 ** 2).sum(1))
            assert (mid == ref_mid).mean() > 0.999
        enc = O.encode(x, means, b1, b2, mean_id=mid)
        assert np.array_equal(got["codes1"].cpu().numpy(), enc["codes1"])
        assert np.array_equal(got["lower"].cpu().numpy().view(np.uint32), enc["lower"].view(np.uint32))
        assert np.array_equal(got["step"].cpu().numpy().view(np.uint32), enc["step"].view(np.uint32))
        if b2:
            assert np.array_equal(got["codes2"].cpu().numpy(), enc["codes2"])
    st.close()


def test_encode_hand_worked_and_degenerate_rows():
    # constant rows (step 0), a row at the quantiser boundary, huge and tiny magnitudes
    d = 16
    rows = [np.zeros(d), np.full(d, 3.25), np.linspace(-1, 1, d), np.linspace(0, 13, d),
            np.r_[np.zeros(d - 1), 1e-30], np.r_[np.full(d - 1, 1e30), -1e30]]
    x = np.array(rows, dtype=np.float32)
    means = np.zeros((1, d), np.float32)
    for b1 in (4, 8):
        st, ids = lib_store(x, means, b1, 8, "l2")
        got = st.encode(torch.from_numpy(x).cuda())
        enc = O.encode(x, means, b1, 8)
        assert np.array_equal(got["codes1"].cpu().numpy(), enc["codes1"])
        assert np.array_equal(got["codes2"].cpu().numpy(), enc["codes2"])
        assert np.array_equal(got["step"].cpu().numpy(), enc["step"])
        assert np.array_equal(got["lower"].cpu().numpy(), enc["lower"])
        st.close()


SEARCH_CASES = [
    # n, d, comps, metric, bits1, bits2, n_means, nq, k1, k
    (10000, 96, 32, "l2", 8, 0, 1, 50, 0, 10),      # LVQ-8 L2, float32 (the 10k x 96 workload)
    (6000, 96, 16, "l2", 4, 8, 1, 40, 50, 10),
    (5000, 768, 32, "ip", 4, 8, 1, 24, 100, 10),
    (4099, 100, 8, "l2", 4, 8, 1, 33, 64, 7),       # ragged n and d
    (3000, 200, 32, "l2", 4, 8, 16, 20, 40, 10),    # M-LVQ L2
    (5000, 768, 64, "ip", 4, 8, 16, 17, 100, 10),   # M-LVQ IP
    (1500, 13, 4, "ip", 8, 8, 1, 5, 30, 30),
    (1500, 4096, 8, "ip", 4, 8, 1, 5, 32, 10),      # the largest d
]


def _s_id(c):
    return "n%d-d%d-%s-%dx%d-M%d-q%d-k%d/%d" % (c[0], c[1], c[3], c[4], c[5], c[6], c[7], c[8], c[9])


@pytest.mark.parametrize("case", SEARCH_CASES, ids=_s_id)
def test_exhaustive_search_fp32(case):
    n, d, comps, metric, b1, b2, m, nq, k1, k = case
    x, q, means = gmm_case(n, d, comps, metric, nq, seed=200 + d, n_means=m)
    st, ids = lib_store(x, means, b1, b2, metric)
    mid = st.export(ids)["mean_id"].cpu().numpy()
    enc = O.encode(x, means, b1, b2, mean_id=mid)
    qt = torch.from_numpy(q).cuda()
    # first level alone
    kk = k1 if k1 else k
    fi, fs = st.first_level(qt, kk, "fp32")
    check_sorted(fs, metric)
    check_scores(q, fi, fs, enc, means, metric, 1, TOL_FP32)
    check_topk_ids(q, fi, fs, enc, means, metric, kk, TOL_FP32, level=1)
    # the whole search
    gi, gs = st.search(qt, k, k1, "fp32")
    check_sorted(gs, metric)
    level = 2 if (b2 and k1) else 1
    check_scores(q, gi, gs, enc, means, metric, level, TOL_FP32)
    if level == 2:
        check_two_level(q, gi, gs, (fi, fs), enc, means, metric, k1, k, TOL_FP32)
    else:
        check_topk_ids(q, gi, gs, enc, means, metric, k, TOL_FP32, level=1)
    st.close()


def test_deletes_are_filtered_and_results_padded():
    x, q, means = gmm_case(3000, 64, 8, "l2", 10, seed=5)
    st, ids = lib_store(x, means, 4, 8, "l2")
    g = np.random.default_rng(0)
    dead = np.unique(g.integers(0, 3000, 1200))
    out = st.delete(torch.from_numpy(dead).cuda())
    assert int(out.item()) == len(dead)
    assert int(st.delete(torch.from_numpy(dead).cuda()).item()) == 0   # idempotent
    live = np.ones(3000, bool)
    live[dead] = False
    assert st.stats() == live.sum()
    enc = O.encode(x, means, 4, 8)
    qt = torch.from_numpy(q).cuda()
    gi, gs = st.search(qt, 10, 40, "fp32")
    assert not np.isin(gi.cpu().numpy(), dead).any()
    check_two_level(q, gi, gs, st.first_level(qt, 40, "fp32"), enc, means, "l2", 40, 10, TOL_FP32, live=live)
    # delete almost everything: fewer live rows than k -> padding
    keep = np.setdiff1d(np.arange(3000), dead)[[0, 7, -1]]
    rest = np.setdiff1d(np.arange(3000), np.r_[dead, keep])
    st.delete(torch.from_numpy(rest).cuda())
    gi, gs = st.search(qt, 10, 40, "fp32")
    gi, gs = gi.cpu().numpy(), gs.cpu().numpy()
    assert np.all(np.sort(gi[:, :3], axis=1) == np.sort(keep)) and np.all(gi[:, 3:] == -1)
    assert np.all(np.isinf(gs[:, 3:])) and np.all(gs[:, 3:] > 0)
    fi, fs = st.first_level(qt, 8, "fp32")
    assert np.all(fi.cpu().numpy()[:, 3:] == -1)
    st.close()


def test_empty_store_and_empty_batch():
    means = np.zeros((1, 32), np.float32)
    from paper_2402_02044_b300 import Store
    st = Store(32, 4, 8, means, "ip", 1000)
    q = torch.randn(3, 32, device="cuda")
    gi, gs = st.search(q, 5, 10, "fp32")
    assert (gi == -1).all() and torch.isinf(gs).all() and (gs < 0).all()
    gi, gs = st.search(q[:0], 5, 10, "fp32")
    assert gi.shape == (0, 5)
    st.close()


@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_candidates_and_rerank(metric):
    n, d, nq, C = 20000, 96, 64, 700
    mix = synth.Mixture(d=d, n_comp=32, sigma=0.3, normalize=metric == "ip", seed=9)
    x, lab = mix.base(n, with_labels=True)
    q, qlab = mix.queries(nq, with_labels=True)
    means = synth.sample_mean(x)[None]
    cand = synth.candidate_lists(lab, qlab, C, 0.7, seed=4)
    cand[:, :5] = -1                       # skipped
    cand[:, 5:9] = cand[:, 9:13]           # repeats
    cand[:, 13] = n + 5                    # out of range
    st, ids = lib_store(x, means, 4, 8, metric)
    dead = cand[:, 20]                     # deleted candidates must vanish
    st.delete(torch.from_numpy(np.unique(dead)).cuda())
    live = np.ones(n, bool)
    live[dead] = False
    enc = O.encode(x, means, 4, 8)
    qt, ct = torch.from_numpy(q).cuda(), torch.from_numpy(cand).cuda()
    gi, gs = st.search_candidates(qt, ct, 10, 50)
    check_sorted(gs, metric)
    check_scores(q, gi, gs, enc, means, metric, 2, TOL_FP32)
    check_two_level(q, gi, gs, st.search_candidates(qt, ct, 50, 0), enc, means, metric, 50, 10, TOL_FP32,
                    live=live, cand_ids=cand)
    # first level only (k1 = 0)
    fi, fs = st.search_candidates(qt, ct, 20, 0)
    check_scores(q, fi, fs, enc, means, metric, 1, TOL_FP32)
    check_topk_ids(q, fi, fs, enc, means, metric, 20, TOL_FP32, live=live, cand_ids=cand)
    # a list holding every live id is the exhaustive search: both forms
    # equal the oracle's exhaustive search, element by element
    allc = torch.from_numpy(np.tile(np.arange(n, dtype=np.int64), (4, 1))).cuda()
    ei, es = st.search(qt[:4], 10, 50, "fp32")
    ai, as_ = st.search_candidates(qt[:4], allc, 10, 50)
    check_two_level(q[:4], ei, es, st.first_level(qt[:4], 50, "fp32"), enc, means, metric, 50, 10, TOL_FP32,
                    live=live)
    check_two_level(q[:4], ai, as_, st.search_candidates(qt[:4], allc, 50, 0), enc, means, metric, 50, 10,
                    TOL_FP32, live=live)
    # rerank of caller-given candidates: the oracle's two-level order of
    # each query's (live, distinct) candidates
    ri, rs = st.rerank(qt, ct[:, :200].contiguous(), 10)
    check_rerank(q, ri, rs, enc, means, metric, cand[:, :200], 10, live=live)
    st.close()


GATHER_CASES = [
    # n, d, comps, metric, bits1, bits2, n_means, nq, C, k1, k
    (20000, 768, 32, "ip", 4, 8, 1, 24, 1000, 100, 10),
    (20000, 768, 32, "l2", 8, 8, 4, 24, 700, 50, 10),
    (6000, 100, 16, "l2", 4, 8, 1, 40, 500, 40, 7),      # ragged d, 16 lanes a candidate
    (3000, 4096, 8, "ip", 4, 8, 1, 6, 300, 30, 10),      # groups beyond the preloaded ones
    (3000, 4096, 8, "l2", 8, 0, 1, 4, 200, 0, 10),       # LVQ-8 single level, largest d
    (4000, 24, 8, "l2", 8, 0, 1, 32, 300, 0, 10),        # 4 lanes a candidate
    (8000, 64, 16, "ip", 4, 8, 256, 32, 600, 60, 10),    # the most centres
    (5000, 96, 16, "ip", 4, 0, 1, 16, 2048, 0, 20),      # many rounds
]


def _gid(c):
    return "n%d-d%d-%s-%dx%d-M%d-C%d-k%d" % (c[0], c[1], c[3], c[4], c[5], c[6], c[8], c[9])


@pytest.mark.parametrize("case", GATHER_CASES, ids=_gid)
def test_candidates_widths_dims_means(case):
    """ID-gather search over code widths, dimensionalities (sub-warp sizes 4
    to 32 lanes, rows longer than the preloaded groups), centring means and
    both metrics: first-level scores within the float32 tolerance, ids equal
    to the oracle's up to near-ties."""
    n, d, comps, metric, b1, b2, m, nq, C, k1, k = case
    x, q, means = gmm_case(n, d, comps, metric, nq, seed=700 + d + m, n_means=m)
    st, ids = lib_store(x, means, b1, b2, metric)
    mid = st.export(ids)["mean_id"].cpu().numpy()
    enc = O.encode(x, means, b1, b2, mean_id=mid)
    g = np.random.default_rng(d + C)
    cand = g.integers(0, n, (nq, C)).astype(np.int64)
    cand[:, 1] = cand[:, 0]          # a repeat
    cand[:, 2] = -1                  # skipped
    qt, ct = torch.from_numpy(q).cuda(), torch.from_numpy(cand).cuda()
    gi, gs = st.search_candidates(qt, ct, k, k1)
    check_sorted(gs, metric)
    if k1 and b2:
        check_scores(q, gi, gs, enc, means, metric, 2, TOL_FP32)
        check_two_level(q, gi, gs, st.search_candidates(qt, ct, k1, 0), enc, means, metric, k1, k, TOL_FP32,
                        cand_ids=cand)
    else:
        check_scores(q, gi, gs, enc, means, metric, 1, TOL_FP32)
        check_topk_ids(q, gi, gs, enc, means, metric, k, TOL_FP32, cand_ids=cand)
    check_no_device_error(st)
    st.close()


def test_candidates_many_queries_per_block_and_limits():
    """More queries than resident gather blocks (each block walks several
    queries, its row ring running across query boundaries), the largest k1,
    a single candidate, the longest candidate list, and lists that are all
    skipped or all deleted."""
    n, d = 6000, 768
    x, q, means = gmm_case(n, d, 16, "ip", 700, seed=77)
    st, ids = lib_store(x, means, 4, 8, "ip")
    enc = O.encode(x, means, 4, 8)
    g = np.random.default_rng(12)
    qt = torch.from_numpy(q).cuda()
    # 700 queries x 90 candidates: several queries per block
    cand = g.integers(0, n, (700, 90)).astype(np.int64)
    gi, gs = st.search_candidates(qt, torch.from_numpy(cand).cuda(), 10, 0)
    check_scores(q, gi, gs, enc, means, "ip", 1, TOL_FP32)
    check_topk_ids(q, gi, gs, enc, means, "ip", 10, TOL_FP32, cand_ids=cand)
    # the largest k1 (512) over 3000 candidates, re-ranked
    c2 = g.integers(0, n, (3, 3000)).astype(np.int64)
    c2t = torch.from_numpy(c2).cuda()
    gi, gs = st.search_candidates(qt[:3], c2t, 20, 512)
    check_scores(q[:3], gi, gs, enc, means, "ip", 2, TOL_FP32)
    check_two_level(q[:3], gi, gs, st.search_candidates(qt[:3], c2t, 512, 0), enc, means, "ip", 512, 20, TOL_FP32,
                    cand_ids=c2)
    # one candidate; the longest list (every id, many times over)
    c3 = g.integers(0, n, (2, 1)).astype(np.int64)
    gi, gs = st.search_candidates(qt[:2], torch.from_numpy(c3).cuda(), 5, 0)
    gi = gi.cpu().numpy()
    assert (gi[:, 0] == c3[:, 0]).all() and (gi[:, 1:] == -1).all()
    c4 = np.tile(np.arange(65536, dtype=np.int64) % n, (2, 1))
    gi, gs = st.search_candidates(qt[:2], torch.from_numpy(c4).cuda(), 10, 0)
    check_topk_ids(q[:2], gi, gs, enc, means, "ip", 10, TOL_FP32)
    # all skipped / all deleted
    c5 = np.full((2, 40), -1, dtype=np.int64)
    gi, gs = st.search_candidates(qt[:2], torch.from_numpy(c5).cuda(), 5, 10)
    assert (gi.cpu().numpy() == -1).all()
    c6 = g.integers(0, n, (2, 40)).astype(np.int64)
    st.delete(torch.from_numpy(np.unique(c6)).cuda())
    gi, gs = st.search_candidates(qt[:2], torch.from_numpy(c6).cuda(), 5, 0)
    assert (gi.cpu().numpy() == -1).all()
    check_no_device_error(st)
    st.close()


def test_candidates_adversarial_query_rounding():
    """A query with one dominant element and every other element tiny and of
    one sign, against vectors whose codes sit far from the code offset: the
    case where rounding the query (the ID-gather first level's integer
    products) errs most.  Scores stay within the float32 tolerance."""
    d = 768
    x = np.zeros((64, d), np.float32)
    x[:, 0] = 15.0
    x[1:, 1:] = np.random.default_rng(2).integers(0, 16, (63, d - 1)).astype(np.float32)
    means = np.zeros((1, d), np.float32)
    q = np.full((2, d), 3e-8, np.float32)
    q[:, 0] = 1.0
    q[1, 1:] = -3e-8
    for metric in ("ip", "l2"):
        st, ids = lib_store(x, means, 4, 8, metric)
        enc = O.encode(x, means, 4, 8)
        cand = np.tile(np.arange(64, dtype=np.int64), (2, 1))
        gi, gs = st.search_candidates(torch.from_numpy(q).cuda(), torch.from_numpy(cand).cuda(), 10, 0)
        check_scores(q, gi, gs, enc, means, metric, 1, TOL_FP32)
        st.close()


def test_streaming_slots_match_the_replay():
    d, cap = 40, 5000
    mix = synth.Mixture(d=d, n_comp=8, sigma=0.3, seed=3)
    x0 = mix.base(4000)
    means = synth.sample_mean(x0)[None]
    st, ids = lib_store(x0, means, 4, 8, "l2", capacity=cap)
    rep = O.SlotReplay(cap)
    assert ids.cpu().tolist() == rep.insert(4000).tolist()
    rows = {i: x0[i] for i in range(4000)}
    g = np.random.default_rng(1)
    for step in range(6):
        live_ids = np.nonzero(rep.live)[0]
        dele = g.choice(live_ids, 300, replace=False)
        dele = np.r_[dele, dele[:5], [-1, cap + 3]]
        n_del = st.delete(torch.from_numpy(dele.astype(np.int64)).cuda())
        assert int(n_del.item()) == rep.delete(dele)
        xn = mix.rows(0, 250 + 20 * step, stream=9) + np.float32(step)
        new = st.insert(torch.from_numpy(xn).cuda())
        ref_new = rep.insert(len(xn))
        assert new.cpu().tolist() == ref_new.tolist()
        for r, v in zip(ref_new, xn):
            rows[int(r)] = v
        assert st.stats() == rep.live.sum()
    # stored records of every live slot are the oracle's encoding of its vector
    live_ids = np.nonzero(rep.live)[0]
    got = st.export(torch.from_numpy(live_ids).cuda())
    enc = O.encode(np.stack([rows[int(i)] for i in live_ids]), means, 4, 8)
    assert np.array_equal(got["codes1"].cpu().numpy(), enc["codes1"])
    assert np.array_equal(got["codes2"].cpu().numpy(), enc["codes2"])
    # a full store refuses an oversized insert as a whole
    free = cap - rep.live.sum()
    bad = st.insert(torch.zeros((free + 1, d), device="cuda"))
    assert (bad == -1).all()
    from paper_2402_02044_b300 import LVQError
    with pytest.raises(LVQError) as e:
        st.stats()
    assert e.value.status == 3
    assert st.stats() == rep.live.sum()
    st.close()

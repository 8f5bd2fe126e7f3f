"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: the expected values come from
hand-worked examples (tests/golden/encode_hand.json), closed forms,
invariants the paper states, textbook special cases, or brute force on tiny
inputs written independently of the oracle's code.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "encode_hand.json")
F32 = np.float32


def _cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


# ---------------------------------------------------------------- hand-worked

@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_hand_worked_encodings(case):
    x = np.array([case["x"]], dtype=F32)
    means = np.array(case["means"], dtype=F32)
    enc = O.encode(x, means, case["bits1"], case["bits2"], grid2=case.get("grid2", "text"))
    assert enc["mean_id"][0] == case["mean_id"]
    assert enc["lower"][0] == F32(case["lower"])
    assert enc["step"][0] == F32(case["step"])
    assert enc["codes1"][0].tolist() == case["codes1"]
    if case["bits2"]:
        assert enc["codes2"][0].tolist() == case["codes2"]
    if "decoded2_minus_x" in case:
        x2 = O.decode_second(enc, means)[0]
        np.testing.assert_allclose(x2 - x[0].astype(np.float64), case["decoded2_minus_x"], rtol=0, atol=1e-15)


@pytest.mark.parametrize("case", [c for c in _cases() if "eps1" in c], ids=lambda c: c["name"])
def test_hand_worked_quantisation_errors(case):
    # Eq. 5 (eps1) and its two-level analogue (eps2), worked by hand: values,
    # not relations, so a squared difference replaced by an absolute one, a
    # centre dropped on both sides or a missing residual term all fail here.
    x = np.array([case["x"]], dtype=F32)
    means = np.array(case["means"], dtype=F32)
    enc = O.encode(x, means, case["bits1"], case["bits2"], grid2=case.get("grid2", "text"))
    assert O.eps_first(x, means, enc) == pytest.approx(case["eps1"], rel=1e-12, abs=1e-300)
    assert O.eps_second(x, means, enc) == pytest.approx(case["eps2"], rel=1e-12, abs=1e-300)


# ------------------------------------------------------------------ invariants

def _gmm(n=3000, d=96, comps=16, normalize=False, seed=7):
    mix = synth.Mixture(d=d, n_comp=comps, sigma=0.3, normalize=normalize, seed=seed)
    x = mix.base(n, threads=1)
    return x, synth.sample_mean(x)


@pytest.mark.parametrize("bits1", [4, 8])
def test_code_range_and_first_level_error(bits1):
    # Eq. 2: codes lie in [0, 2^B - 1] and each component of the centred
    # reconstruction is within D/2 of the centred input.
    x, mu = _gmm()
    enc = O.encode(x, mu[None], bits1, 8)
    assert enc["codes1"].max() <= (1 << bits1) - 1 and enc["codes2"].max() <= 255
    y = x.astype(np.float64) - mu.astype(np.float64)[None]
    yhat = enc["lower"].astype(np.float64)[:, None] + enc["step"].astype(np.float64)[:, None] * enc["codes1"]
    slack = np.spacing(np.abs(y).max(axis=1).astype(F32)).astype(np.float64) * 4
    assert np.all(np.abs(y - yhat) <= enc["step"][:, None] / 2 + slack[:, None])


def test_decoded_min_and_max_match_bounds():
    # Eq. 1: l(x) = min_j (x_j - mu_j) is reproduced exactly by code 0;
    # u(x) by the top code up to two ulps of |u| + |l| (the step and the
    # reconstruction are rounded).
    x, mu = _gmm()
    for bits1 in (4, 8):
        enc = O.encode(x, mu[None], bits1)
        y = (x - mu[None]).astype(F32)
        yhat = (enc["step"][:, None] * enc["codes1"].astype(F32)).astype(F32) + enc["lower"][:, None]
        assert np.array_equal(yhat.min(axis=1), y.min(axis=1))
        assert np.array_equal(enc["lower"], y.min(axis=1))
        u = y.max(axis=1)
        ulp = np.spacing((np.abs(u) + np.abs(enc["lower"])).astype(F32))
        assert np.all(np.abs(yhat.max(axis=1) - u) <= 2 * ulp)
        assert np.all(enc["codes1"].max(axis=1) == (1 << bits1) - 1)


def test_residual_level_tightens_error():
    # Sec. 2.2: r = x - mu - Q(x) lies in [-D/2, D/2]; its B2-bit code is
    # within D2/2 of it, and the two-level error is below the first-level one.
    x, mu = _gmm()
    enc = O.encode(x, mu[None], 4, 8)
    y = x.astype(np.float64) - mu.astype(np.float64)[None]
    x1 = O.decode_first(enc, mu[None]) - mu.astype(np.float64)[None]
    r = y - x1
    lower2, step2 = O.residual_grid(enc["step"], 8)
    rhat = lower2.astype(np.float64)[:, None] + step2.astype(np.float64)[:, None] * enc["codes2"]
    slack = np.spacing(np.abs(y).max(axis=1).astype(F32)).astype(np.float64) * 4
    assert np.all(np.abs(r) <= enc["step"][:, None] / 2 + slack[:, None])
    assert np.all(np.abs(r - rhat) <= step2[:, None] / 2 + slack[:, None])
    e1, e2 = O.eps_first(x, mu[None], enc), O.eps_second(x, mu[None], enc)
    assert e2 < e1 / 100


@pytest.mark.parametrize("bits1,bits2,grid2", [(2, 8, "text"), (3, 8, "text"), (5, 4, "text"), (6, 2, "text"),
                                               (7, 3, "text"), (8, 2, "text"), (4, 8, "listing"),
                                               (8, 2, "listing"), (3, 5, "listing")])
def test_other_widths_code_ranges_and_error_bounds(bits1, bits2, grid2):
    # Sec. 3.3 (B1, B2 heatmap) and App. C: for every width the first-level
    # codes lie in [0, 2^B1 - 1] and err by at most D/2; the residual codes
    # lie on their grid and err by at most D2/2 (text grid) or D2/2 inside the
    # signed grid's range and D2 at its clipped top (listing grid); the two
    # levels together err less than the first level alone.
    x, mu = _gmm(n=1500)
    enc = O.encode(x, mu[None], bits1, bits2, grid2=grid2)
    assert enc["codes1"].max() <= (1 << bits1) - 1 and enc["codes1"].min() >= 0
    y = x.astype(np.float64) - mu.astype(np.float64)[None]
    x1 = O.decode_first(enc, mu[None]) - mu.astype(np.float64)[None]
    slack = np.spacing(np.abs(y).max(axis=1).astype(F32)).astype(np.float64)[:, None] * 8
    assert np.all(np.abs(y - x1) <= enc["step"][:, None] / 2 + slack)
    r = y - x1
    lower2, step2 = O.residual_grid(enc["step"], bits2, grid2)
    c2 = enc["codes2"].astype(np.int64)
    rhat = lower2.astype(np.float64)[:, None] + step2.astype(np.float64)[:, None] * c2
    if grid2 == "text":
        assert c2.min() >= 0 and c2.max() <= (1 << bits2) - 1
        assert np.all(np.abs(r - rhat) <= step2[:, None] / 2 + slack)
    else:
        half = 1 << (bits2 - 1)
        assert c2.min() >= -half and c2.max() <= half - 1
        # r lies in [-D/2, D/2] = [-half D2, half D2]: only the top code clips
        bound = np.where(c2 == half - 1, step2[:, None], step2[:, None] / 2)
        assert np.all(np.abs(r - rhat) <= bound + slack)
    assert O.eps_second(x, mu[None], enc) < O.eps_first(x, mu[None], enc)


def test_uniform_quantiser_mean_square_error():
    # Textbook uniform quantiser: for inputs spread evenly over a cell the
    # mean squared error is D^2/12.
    g = np.random.default_rng(3)
    x = g.uniform(-1, 1, size=(4000, 256)).astype(F32)
    enc = O.encode(x, np.zeros((1, 256), F32), 4)
    y = x.astype(np.float64)
    yhat = enc["lower"].astype(np.float64)[:, None] + enc["step"].astype(np.float64)[:, None] * enc["codes1"]
    mse = ((y - yhat) ** 2).mean(axis=1)
    expected = enc["step"].astype(np.float64) ** 2 / 12
    assert abs(mse.mean() / expected.mean() - 1) < 0.05


def test_eight_bits_refine_the_step_by_seventeen():
    # D = (u - l)/(2^B - 1): going from 4 to 8 bits divides it by 255/15 = 17.
    x, mu = _gmm(n=500)
    e4 = O.encode(x, mu[None], 4)
    e8 = O.encode(x, mu[None], 8)
    np.testing.assert_allclose(e4["step"] / e8["step"], 17.0, rtol=1e-6)


def test_single_mean_is_plain_lvq_and_more_means_reduce_error():
    # Sec. 3.2: M = 1 is LVQ; Eq. 5 / Def. 1: with centres fitted to a
    # mixture the first-level error drops.
    mix = synth.Mixture(d=64, n_comp=16, sigma=0.3, seed=11)
    x = mix.base(4000, threads=1)
    mu = synth.sample_mean(x)
    e_lvq = O.encode(x, mu[None], 4)
    e_one = O.encode(x, mu[None], 4, mean_id=np.zeros(len(x), np.uint8))
    assert all(np.array_equal(e_lvq[k], e_one[k]) for k in ("codes1", "lower", "step"))
    cen = synth.kmeans_means(x, 16, seed=5)
    e_m = O.encode(x, cen, 4)
    assert O.eps_first(x, cen, e_m) < 0.5 * O.eps_first(x, mu[None], e_lvq)


def test_assignment_is_the_nearest_centre_by_brute_force():
    g = np.random.default_rng(5)
    x = g.standard_normal((200, 8)).astype(F32)
    cen = g.standard_normal((7, 8)).astype(F32)
    m = O.assign_means(x, cen)
    for i in range(len(x)):
        d = [sum((float(x[i, j]) - float(cen[c, j])) ** 2 for j in range(8)) for c in range(7)]
        assert m[i] == d.index(min(d))


# ------------------------------------------------------------------- scoring

def test_scores_match_the_factorised_forms():
    # Sec. 3.2: <q, x^> = <q, mu_m> + l * sum(q) + D * <q, c> and
    # ||q - x^||^2 = ||q_m||^2 - 2 <q_m, Q(x)> + ||Q(x)||^2 with q_m = q - mu_m.
    mix = synth.Mixture(d=48, n_comp=8, sigma=0.3, seed=2)
    x = mix.base(300, threads=1)
    q = mix.queries(5, threads=1)
    cen = synth.kmeans_means(x, 4, seed=1)
    enc = O.encode(x, cen, 4, 8)
    q64, c = q.astype(np.float64), enc["codes1"].astype(np.float64)
    lo, st = enc["lower"].astype(np.float64), enc["step"].astype(np.float64)
    mu = cen.astype(np.float64)[enc["mean_id"].astype(int)]
    ip = np.einsum("qd,nd->qn", q64, mu)  # <q, mu_m(i)>
    ip = ip + lo[None] * q64.sum(1)[:, None] + st[None] * (q64 @ c.T)
    np.testing.assert_allclose(O.score(q, O.decode_first(enc, cen), O.IP), ip, rtol=1e-12, atol=1e-12)
    qm = q64[:, None, :] - mu[None]                      # [nq, n, d]
    qx = lo[None] * qm.sum(-1) + st[None] * np.einsum("qnd,nd->qn", qm, c)
    qq = (qm ** 2).sum(-1)
    xx = (lo[:, None] + st[:, None] * c)
    l2 = qq - 2 * qx + (xx ** 2).sum(-1)[None]
    np.testing.assert_allclose(O.score(q, O.decode_first(enc, cen), O.L2), l2, rtol=1e-10, atol=1e-9)


def test_on_grid_data_decodes_exactly_and_scores_are_plain():
    # Vectors already on an 8-bit grid (x = mu + l + D*c with both end codes
    # present and D a power of two) decode to themselves; the search then
    # reduces to a plain dot product / squared distance.
    g = np.random.default_rng(9)
    n, d = 64, 32
    c = g.integers(0, 256, size=(n, d))
    c[:, 0], c[:, 1] = 0, 255
    lo = g.integers(-8, 8, size=n).astype(np.float64)
    step = 2.0 ** g.integers(-6, -2, size=n)
    mu = np.zeros(d, F32)
    x = (lo[:, None] + step[:, None] * c).astype(F32)
    enc = O.encode(x, mu[None], 8)
    assert np.array_equal(enc["codes1"], c)
    np.testing.assert_array_equal(O.decode_first(enc, mu[None]), x.astype(np.float64))
    q = g.standard_normal((3, d)).astype(F32)
    np.testing.assert_allclose(O.score(q, O.decode_first(enc, mu[None]), O.IP), q.astype(np.float64) @ x.T.astype(np.float64), rtol=1e-13)
    ref = np.array([[np.sum((q[i].astype(np.float64) - x[j]) ** 2) for j in range(n)] for i in range(3)])
    np.testing.assert_allclose(O.score(q, O.decode_first(enc, mu[None]), O.L2), ref, rtol=1e-13)


# ------------------------------------------------------------------ selection

def _brute_topk(scores, ids, k, metric):
    pairs = sorted(zip(scores.tolist(), ids.tolist()),
                   key=(lambda p: (p[0], p[1])) if metric == O.L2 else (lambda p: (-p[0], p[1])))
    return [p[1] for p in pairs[:k]]


@pytest.mark.parametrize("metric", [O.L2, O.IP])
def test_search_matches_brute_force_with_ties_and_deletes(metric):
    g = np.random.default_rng(17)
    n, d = 64, 16
    x = g.integers(-2, 3, size=(n, d)).astype(F32)     # small integers: many ties
    x[:, 0], x[:, 1] = -2, 2
    mu = np.zeros((1, d), F32)
    enc = O.encode(x, mu, 8)
    live = g.random(n) > 0.25
    q = g.integers(-2, 3, size=(4, d)).astype(F32)
    ids, s = O.search_exhaustive(enc, mu, q, 0, 10, metric, live)
    xhat = O.decode_first(enc, mu)
    alive = np.nonzero(live)[0]
    for i in range(len(q)):
        sc = np.array([float(np.dot(q[i].astype(np.float64), xhat[j])) if metric == O.IP
                       else float(np.sum((q[i].astype(np.float64) - xhat[j]) ** 2)) for j in alive])
        assert ids[i].tolist() == _brute_topk(sc, alive, 10, metric)
    # permuting the database rows changes the ids (and so the order among
    # equal scores) but not the scores returned, and every returned row
    # keeps its score
    perm = g.permutation(n)
    enc_p = O.take(enc, perm)
    ids_p, s_p = O.search_exhaustive(enc_p, mu, q, 0, 10, metric, live[perm])
    assert np.array_equal(s_p, s)
    full = O.score(q, xhat, metric)
    for i in range(len(q)):
        assert np.array_equal(full[i, perm[ids_p[i]]], s[i])


def test_padding_when_fewer_live_than_k():
    x = np.eye(4, dtype=F32)
    mu = np.zeros((1, 4), F32)
    enc = O.encode(x, mu, 8, 8)
    live = np.array([True, False, True, False])
    ids, s = O.search_exhaustive(enc, mu, x[:1], 4, 3, O.L2, live)
    assert ids[0].tolist()[2] == -1 and s[0, 2] == np.inf
    ids, s = O.search_exhaustive(enc, mu, x[:1], 4, 3, O.IP, live)
    assert ids[0].tolist()[2] == -1 and s[0, 2] == -np.inf


def test_rerank_uses_two_levels_and_gather_equals_exhaustive():
    mix = synth.Mixture(d=32, n_comp=4, sigma=0.3, seed=4)
    x = mix.base(500, threads=1)
    q = mix.queries(6, threads=1)
    mu = synth.sample_mean(x)[None]
    enc = O.encode(x, mu, 4, 8)
    ids, s = O.search_exhaustive(enc, mu, q, 40, 10, O.L2)
    # stage 1 by hand: k1 best first-level ids, then second-level order
    s1 = O.score(q, O.decode_first(enc, mu), O.L2)
    s2 = O.score(q, O.decode_second(enc, mu), O.L2)
    for i in range(len(q)):
        cand = np.array(_brute_topk(s1[i], np.arange(500), 40, O.L2))
        assert ids[i].tolist() == [int(v) for v in cand[np.array(_brute_topk(s2[i][cand], np.arange(40), 10, O.L2))]]
    # the ID-gather form with every id (shuffled, with -1 and repeats) is the same search
    g = np.random.default_rng(1)
    cand = np.stack([np.concatenate([g.permutation(500), [-1, -1, 3, 499]]) for _ in q])
    ids_c, s_c = O.search_candidates(enc, mu, q, cand, 40, 10, O.L2)
    assert np.array_equal(ids_c, ids) and np.array_equal(s_c, s)
    gt, _ = O.ground_truth(enc, mu, q, 10, O.L2)
    for i in range(len(q)):
        assert gt[i].tolist() == _brute_topk(s2[i], np.arange(500), 10, O.L2)


@pytest.mark.parametrize("metric", [O.L2, O.IP])
def test_exact_knn_of_raw_vectors_by_brute_force(metric):
    # Sec. 2.1: the k nearest by the raw vectors, ties to the lower id
    g = np.random.default_rng(23)
    x = g.integers(-3, 4, size=(40, 6)).astype(F32)
    q = g.integers(-3, 4, size=(3, 6)).astype(F32)
    ids, s = O.exact_knn(x, q, 7, metric, chunk=16)
    for i in range(len(q)):
        sc = np.array([sum(float(q[i, j]) * float(x[r, j]) for j in range(6)) if metric == O.IP
                       else sum((float(q[i, j]) - float(x[r, j])) ** 2 for j in range(6)) for r in range(40)])
        assert ids[i].tolist() == _brute_topk(sc, np.arange(40), 7, metric)
        assert s[i].tolist() == [sc[r] for r in ids[i]]


def test_recall_at_k():
    assert O.recall_at_k(np.array([[1, 2, 3, 4]]), np.array([[4, 3, 9, 8]]), 4) == 0.5
    assert O.recall_at_k(np.array([[1, -1]]), np.array([[1, 2]]), 2) == 0.5


# ------------------------------------------------------------------- the store

def test_slot_replay_policy_by_brute_force():
    rep = O.SlotReplay(10)
    assert rep.insert(4).tolist() == [0, 1, 2, 3]
    assert rep.delete([2, 2, 0, 17, -1, 5]) == 2
    assert rep.insert(3).tolist() == [0, 2, 4]
    with pytest.raises(O.StoreFull):
        rep.insert(6)
    assert rep.live.sum() == 5
    assert rep.insert(5).tolist() == [5, 6, 7, 8, 9]


# --------------------------------------------------- the pins catch mistakes

def test_planted_mistakes_are_caught(monkeypatch):
    """Each planted mistake in the oracle makes one of the pins above fail."""
    case = _cases()[4]   # round half up
    x = np.array([case["x"]], F32)
    means = np.array(case["means"], F32)

    def half_even(v, lower, step, bits):
        step_c = np.where(step == 0, F32(1), step).astype(F32)
        t = ((F32(1) / step_c)[:, None] * (v - lower[:, None]).astype(F32)).astype(F32)
        return np.clip(np.round(t), 0, (1 << bits) - 1).astype(np.uint8)
    monkeypatch.setattr(O.lvq, "quantize", half_even)
    assert O.encode(x, means, 2)["codes1"][0].tolist() != case["codes1"]
    monkeypatch.undo()

    def div_form(v, lower, step, bits):
        step_c = np.where(step == 0, F32(1), step).astype(F32)
        t = (((v - lower[:, None]).astype(F32) / step_c[:, None]).astype(F32) + F32(0.5)).astype(F32)
        return np.clip(np.floor(t), 0, (1 << bits) - 1).astype(np.uint8)
    c1 = _cases()[1]     # reciprocal form
    monkeypatch.setattr(O.lvq, "quantize", div_form)
    assert O.encode(np.array([c1["x"]], F32), np.array(c1["means"], F32), 2)["codes1"][0].tolist() != c1["codes1"]
    monkeypatch.undo()

    # eps with absolute instead of squared differences, or with the centre
    # dropped from both the vector and its reconstruction, misses the
    # hand-worked value of Eq. 5
    ce = [c for c in _cases() if c["name"].startswith("non-zero first-level")][0]
    xe, me = np.array([ce["x"]], F32), np.array(ce["means"], F32)
    enc_e = O.encode(xe, me, ce["bits1"], ce["bits2"])
    x1 = O.decode_first(enc_e, me)
    abs_sum = float(np.abs(xe.astype(np.float64) - x1).sum())
    no_centre = float(((xe.astype(np.float64) - (x1 - me.astype(np.float64))) ** 2).sum())
    assert abs_sum != pytest.approx(ce["eps1"]) and no_centre != pytest.approx(ce["eps1"])
    assert O.eps_first(xe, me, enc_e) == pytest.approx(ce["eps1"])

    # a decode that forgets the centre breaks the inner-product factorisation
    mix = synth.Mixture(d=16, n_comp=4, sigma=0.3, seed=3)
    xx = mix.base(50, threads=1)
    mu = synth.sample_mean(xx)[None] + F32(1)
    enc = O.encode(xx, mu, 4)
    good = O.decode_first(enc, mu)
    bad = good - mu.astype(np.float64)
    q = mix.queries(2, threads=1).astype(np.float64)
    fact = q @ mu.astype(np.float64)[0][:, None] + enc["lower"][None] * q.sum(1)[:, None] \
        + enc["step"][None] * (q @ enc["codes1"].T.astype(np.float64))
    assert np.allclose(q @ good.T, fact) and not np.allclose(q @ bad.T, fact)


# ---- M-LVQ centre update (Sec. 3.2) -------------------------------------------

def _on_grid_store():
    """Two integer centres and rows x = mu_m + l + c with integer l and codes
    c in [0, 15] (0 and 15 present in each row): every float32 step is exact."""
    g = np.random.default_rng(11)
    d, n = 12, 40
    means = g.integers(-20, 20, (2, d)).astype(F32)
    m = np.arange(n) % 2
    lower = g.integers(-9, 9, n).astype(F32)
    c = g.integers(0, 16, (n, d))
    c[:, 0], c[:, 1] = 0, 15
    x = (means[m] + lower[:, None] + c).astype(F32)
    return x, means, m.astype(np.uint8), c


def test_update_mean_by_a_constant_shift_is_exact():
    x, means, m, c = _on_grid_store()
    enc = O.encode(x, means, 4, mean_id=m)
    assert np.array_equal(enc["codes1"], c) and np.all(enc["step"] == 1)
    shifted = means[1] + F32(3)
    new, means2, cnt = O.update_mean(enc, means, 1, shifted)
    t = m == 1
    assert cnt == t.sum()
    # codes and steps kept, lower bounds down by 3, the same vectors decoded
    assert np.array_equal(new["codes1"], enc["codes1"]) and np.array_equal(new["step"], enc["step"])
    assert np.array_equal(new["lower"][t], enc["lower"][t] - 3) and np.array_equal(new["lower"][~t], enc["lower"][~t])
    assert np.array_equal(O.decode_first(new, means2), O.decode_first(enc, means))
    # a mistaken update that reconstructs with the new centre decodes elsewhere
    wrong = O.encode(O.reconstruct_f32(enc, means2), means2, 4, mean_id=m)
    assert not np.array_equal(O.decode_first(wrong, means2)[t], O.decode_first(enc, means)[t])


def test_reconstruct_f32_is_the_float64_decode_up_to_rounding():
    mix = synth.Mixture(d=40, n_comp=4, sigma=0.3, seed=5)
    x = mix.base(300, threads=1)
    means = synth.kmeans_means(x, 3, seed=5, iters=5)
    enc = O.encode(x, means, 4, 8)
    r = O.reconstruct_f32(enc, means).astype(np.float64)
    ref = O.decode_second(enc, means)
    assert np.all(np.abs(r - ref) <= 4 * np.finfo(np.float32).eps * (np.abs(ref) + 1))


def test_update_mean_re_encodes_only_live_tagged_rows_within_the_bound():
    mix = synth.Mixture(d=40, n_comp=4, sigma=0.3, seed=6)
    x = mix.base(400, threads=1)
    means = synth.kmeans_means(x, 3, seed=6, iters=5)
    enc = O.encode(x, means, 4, 8)
    live = np.ones(400, bool)
    live[::7] = False
    m = int(np.bincount(enc["mean_id"]).argmax())
    new_mu = means[m] + F32(0.05) * np.sin(np.arange(40, dtype=F32))
    before = O.reconstruct_f32(enc, means)
    new, means2, cnt = O.update_mean(enc, means, m, new_mu, live=live)
    t = live & (enc["mean_id"] == m)
    assert cnt == t.sum() > 0 and np.array_equal(new["mean_id"], enc["mean_id"])
    for key in ("codes1", "codes2", "lower", "step"):
        assert np.array_equal(new[key][~t], enc[key][~t])
    # the re-encoded two-level decode is within half a residual step of the
    # reconstruction it was encoded from (plus float rounding)
    _, step2 = O.residual_grid(new["step"][t], 8)
    err = np.abs(O.decode_second(O.take(new, np.nonzero(t)[0]), means2) - before[t])
    assert np.all(err <= step2[:, None] / 2 * (1 + 1e-4) + 1e-6)


# ---- greedy beam search (Alg. 1) ---------------------------------------------

def test_beam_search_on_a_complete_graph_is_the_exhaustive_search():
    mix = synth.Mixture(d=16, n_comp=4, sigma=0.3, seed=8)
    x = mix.base(60, threads=1)
    means = synth.sample_mean(x)[None]
    enc = O.encode(x, means, 4)
    q = mix.queries(3, threads=1)
    graph = np.array([[j for j in range(60) if j != i] for i in range(60)])
    live = np.ones(60, bool)
    live[[3, 17]] = False
    for metric in ("l2", "ip"):
        bi, bs = O.beam_search(enc, means, q, graph, [0], L=60, k=10, metric=metric, live=live)
        ei, es = O.search_exhaustive(enc, means, q, 0, 10, metric, live=live)
        assert np.array_equal(bi, ei) and np.allclose(bs, es)


def test_beam_search_follows_the_graph():
    # a path 0 - 1 - ... - 9 in one dimension, query beyond node 9: from node
    # 0 with L = 2 the search walks the path and ends at the far end; with no
    # expansions it returns the start
    x = np.arange(10, dtype=F32)[:, None] * np.ones((1, 8), F32)
    means = np.zeros((1, 8), F32)
    enc = O.encode(x, means, 8)
    q = np.full((1, 8), 20.0, F32)
    graph = np.array([[max(i - 1, 0), min(i + 1, 9)] for i in range(10)])
    ids, _ = O.beam_search(enc, means, q, graph, [0], L=2, k=2, metric="l2")
    assert ids[0].tolist() == [9, 8]
    ids, _ = O.beam_search(enc, means, q, graph, [0], L=2, k=2, metric="l2", max_expand=0)
    assert ids[0].tolist() == [0, -1]

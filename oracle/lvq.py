"""Plain CPU restatement of LVQ encoding and brute-force LVQ search.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every float32 step is
written as its own numpy operation on float32 arrays, so each one is rounded
once, in the order given here; numpy never fuses a multiply and an add.
Decoding and scoring are carried out in float64.

Readings of points the paper leaves open (each one is also listed with its
reason in the design notes of the repository):

* (i)   the quantiser multiplies by a rounded reciprocal of the step instead
        of dividing by it, as the paper's listing does (App. C); Eq. 2 writes
        a division.
* (ii)  rounding is floor(t + 1/2) (Eq. 2) at both levels.
* (iii) the second level uses the text's grid Q_{B2,-Delta/2,Delta/2}
        (Sec. 2.2, Def. 1): unsigned codes, step Delta/(2^B2 - 1).  The App. C
        listing's signed grid (step Delta/2^B2, codes rounded half to even and
        clipped to [-2^(B2-1), 2^(B2-1) - 1], no offset) is the option
        grid2="listing".
* (iv)  a constant centred vector (Delta = 0) is coded with a unit step
        (all codes 0, as in App. C) but Delta = 0 is stored, so it decodes
        exactly.
* (v)   u(x) = max_j (x_j - mu_j), l(x) = min_j (x_j - mu_j) (Eq. 1).
* (vi)  the centring means are inputs.
* (vii) the M-LVQ centre is the float64 argmin, lowest index on ties.
* (viii) the inner product with M-LVQ is <q, Q(x)> + <q, mu_m> (Sec. 3.2).
* (ix)  "L2" results are squared Euclidean distances.
* (xii) results are ordered by (score, id): ascending distance or
        descending inner product, the lower id first on equal scores.
"""
from __future__ import annotations

import numpy as np

F32 = np.float32
F64 = np.float64

L2 = "l2"
IP = "ip"

__all__ = [
    "L2", "IP", "assign_means", "quantize", "residual_grid", "encode", "decode_first",
    "decode_second", "decode", "score", "best_first", "topk", "search_exhaustive",
    "search_candidates", "rerank", "ground_truth", "recall_at_k", "eps_first", "eps_second",
    "SlotReplay", "StoreFull", "pad_value", "take", "first_level_candidates", "quantize_signed",
    "reconstruct_f32", "update_mean", "beam_search", "exact_knn",
]


# --------------------------------------------------------------------------
# Encoding: Eq. 1-3, Sec. 2.2 and Def. 1
# --------------------------------------------------------------------------

def assign_means(x: np.ndarray, means: np.ndarray) -> np.ndarray:
    """Def. 1: index of the centre nearest to each row, argmin_m ||x - mu_m||^2.

    The squared distances are summed in float64 from the float32 inputs; the
    lowest index wins a tie (np.argmin returns the first minimum).  With a
    single centre every row gets index 0 (M = 1 is plain LVQ, Sec. 3.2)."""
    x = np.asarray(x, dtype=F32)
    means = np.asarray(means, dtype=F32).reshape(-1, x.shape[1])
    if len(means) == 1:
        return np.zeros(len(x), dtype=np.uint8)
    x64 = x.astype(F64)
    dist = np.empty((len(x), len(means)), dtype=F64)
    for m in range(len(means)):
        diff = x64 - means[m].astype(F64)[None, :]
        dist[:, m] = (diff * diff).sum(axis=1)
    return np.argmin(dist, axis=1).astype(np.uint8)


def quantize(v: np.ndarray, lower: np.ndarray, step: np.ndarray, bits: int) -> np.ndarray:
    """Codes of the scalar quantiser Q_{B,l,u} of Eq. 2, one row per vector.

    code = clip(floor(inv * (v - l) + 1/2), 0, 2^B - 1) with inv = 1/step,
    each operation rounded to float32 (reading (i), (ii)).  A zero step is
    replaced by 1 for the code computation only (reading (iv))."""
    v = np.asarray(v, dtype=F32)
    lower = np.asarray(lower, dtype=F32)
    step = np.asarray(step, dtype=F32)
    step_c = np.where(step == F32(0), F32(1), step).astype(F32)
    inv = (F32(1) / step_c).astype(F32)
    shifted = (v - lower[:, None]).astype(F32)
    scaled = (inv[:, None] * shifted).astype(F32)
    t = (scaled + F32(0.5)).astype(F32)
    codes = np.floor(t)
    return np.clip(codes, 0, (1 << bits) - 1).astype(np.uint8)


def residual_grid(step: np.ndarray, bits2: int, grid2: str = "text"):
    """Lower bound and step of the second-level quantiser.

    "text": Q_{B2,-D/2,D/2} (Sec. 2.2, Def. 1): l2 = -step/2 (exact) and
    step2 = step/(2^B2 - 1), rounded to float32.
    "listing": the signed grid of App. C: l2 = 0, step2 = step/2^B2 (a power
    of two: exact)."""
    step = np.asarray(step, dtype=F32)
    if grid2 == "listing":
        return np.zeros_like(step), (step / F32(1 << bits2)).astype(F32)
    lower2 = (-step * F32(0.5)).astype(F32)
    step2 = (step / F32((1 << bits2) - 1)).astype(F32)
    return lower2, step2


def quantize_signed(v: np.ndarray, step: np.ndarray, bits: int) -> np.ndarray:
    """The App. C listing's residual codes: round(v * (1/step)) half to even,
    clipped to [-2^(B-1), 2^(B-1) - 1], in float32 (a zero step is replaced
    by 1 for the codes)."""
    v = np.asarray(v, dtype=F32)
    step = np.asarray(step, dtype=F32)
    step_c = np.where(step == F32(0), F32(1), step).astype(F32)
    inv = (F32(1) / step_c).astype(F32)
    t = (inv[:, None] * v).astype(F32)
    half = 1 << (bits - 1)
    return np.clip(np.round(t), -half, half - 1).astype(np.int8)


def encode(x: np.ndarray, means: np.ndarray, bits1: int, bits2: int = 0, mean_id=None, grid2: str = "text") -> dict:
    """LVQ-B1 or LVQ-B1xB2 of each row of ``x`` (M-LVQ when several means).

    Steps: nearest centre (Def. 1) -> centred y = x - mu* (float32) ->
    bounds u = max y, l = min y (Eq. 1) -> step D = (u - l)/(2^B1 - 1)
    (Eq. 2) -> first-level codes (Eq. 2, 3) -> centred reconstruction
    y^ = D*c + l -> residual r = y - y^ (Sec. 2.2) -> second-level codes of r
    on the grid of ``residual_grid`` (``grid2``: "text" or "listing").

    Returns a dict with ``codes1`` [n, d] uint8 (one code per byte),
    ``codes2`` [n, d] (uint8 on the text grid, int8 on the listing's) or
    None, ``lower`` and ``step`` float32 [n], ``mean_id`` uint8 [n], the bit
    widths and the residual grid."""
    x = np.asarray(x, dtype=F32)
    means = np.asarray(means, dtype=F32).reshape(-1, x.shape[1])
    m = assign_means(x, means) if mean_id is None else np.asarray(mean_id, dtype=np.uint8)
    y = (x - means[m.astype(np.int64)]).astype(F32)
    u = y.max(axis=1)
    lower = y.min(axis=1)
    step = ((u - lower).astype(F32) / F32((1 << bits1) - 1)).astype(F32)
    codes1 = quantize(y, lower, step, bits1)
    y_hat = ((step[:, None] * codes1.astype(F32)).astype(F32) + lower[:, None]).astype(F32)
    out = dict(codes1=codes1, codes2=None, lower=lower, step=step, mean_id=m,
               bits1=bits1, bits2=bits2, grid2=grid2)
    if bits2:
        r = (y - y_hat).astype(F32)
        lower2, step2 = residual_grid(step, bits2, grid2)
        out["codes2"] = quantize_signed(r, step2, bits2) if grid2 == "listing" else quantize(r, lower2, step2, bits2)
    return out


def take(enc: dict, rows) -> dict:
    """The encoded records of the given row indices."""
    rows = np.asarray(rows, dtype=np.int64)
    out = dict(enc)
    for key in ("codes1", "codes2", "lower", "step", "mean_id"):
        if enc.get(key) is not None:
            out[key] = enc[key][rows]
    return out


# --------------------------------------------------------------------------
# Decoding (float64, from the stored representation)
# --------------------------------------------------------------------------

def decode_first(enc: dict, means: np.ndarray) -> np.ndarray:
    """x^1 = mu_m + l + D * c  (Sec. 3.2: x ~ Q(x) + mu), float64 [n, d]."""
    means = np.asarray(means, dtype=F32).reshape(-1, enc["codes1"].shape[1]).astype(F64)
    mu = means[enc["mean_id"].astype(np.int64)]
    return mu + enc["lower"].astype(F64)[:, None] + enc["step"].astype(F64)[:, None] * enc["codes1"].astype(F64)


def decode_second(enc: dict, means: np.ndarray) -> np.ndarray:
    """x^2 = x^1 + l2 + D2 * c2: first level plus the decoded residual."""
    x1 = decode_first(enc, means)
    if not enc.get("bits2"):
        return x1
    lower2, step2 = residual_grid(enc["step"], enc["bits2"], enc.get("grid2", "text"))
    return x1 + lower2.astype(F64)[:, None] + step2.astype(F64)[:, None] * enc["codes2"].astype(F64)


def decode(enc: dict, means: np.ndarray, level: int) -> np.ndarray:
    return decode_first(enc, means) if level == 1 else decode_second(enc, means)


# --------------------------------------------------------------------------
# Scoring and selection
# --------------------------------------------------------------------------

def score(q: np.ndarray, xhat: np.ndarray, metric: str) -> np.ndarray:
    """Scores of every query against every decoded row, float64 [nq, n].

    L2: sum_j (q_j - x_j)^2 (squared Euclidean distance, lower is better).
    IP: sum_j q_j x_j (inner product, higher is better)."""
    q = np.atleast_2d(np.asarray(q)).astype(F64)
    xhat = np.asarray(xhat, dtype=F64)
    if metric == IP:
        return q @ xhat.T
    out = np.empty((len(q), len(xhat)), dtype=F64)
    for i in range(len(q)):
        diff = xhat - q[i][None, :]
        out[i] = (diff * diff).sum(axis=1)
    return out


def best_first(scores: np.ndarray, ids: np.ndarray, metric: str) -> np.ndarray:
    """Permutation that orders (score, id) pairs best first, ties by lower id."""
    key = scores if metric == L2 else -scores
    return np.lexsort((ids, key))


def pad_value(metric: str) -> float:
    return np.inf if metric == L2 else -np.inf


def topk(scores: np.ndarray, ids: np.ndarray, k: int, metric: str):
    """The k best (id, score) pairs of one query, padded with (-1, +/-inf)."""
    order = best_first(scores, ids, metric)[:k]
    out_ids = np.full(k, -1, dtype=np.int64)
    out_s = np.full(k, pad_value(metric), dtype=F64)
    out_ids[:len(order)] = ids[order]
    out_s[:len(order)] = scores[order]
    return out_ids, out_s


def _live_ids(live) -> np.ndarray:
    return np.nonzero(np.asarray(live, dtype=bool))[0].astype(np.int64)


def rerank(enc: dict, means, q, ids, k: int, metric: str, live=None):
    """Residual re-ranking (Sec. 2.2, App. C): reorder each query's candidate
    ids by the two-level score and keep k.  Ids that are negative, out of
    range, repeated or not live are dropped."""
    q = np.atleast_2d(np.asarray(q, dtype=F32))
    ids = np.atleast_2d(np.asarray(ids, dtype=np.int64))
    n = len(enc["lower"])
    live = np.ones(n, dtype=bool) if live is None else np.asarray(live, dtype=bool)
    out_ids = np.full((len(q), k), -1, dtype=np.int64)
    out_s = np.full((len(q), k), pad_value(metric), dtype=F64)
    for i in range(len(q)):
        c = ids[i]
        c = c[(c >= 0) & (c < n)]
        c = np.unique(c)
        c = c[live[c]]
        if len(c) == 0:
            continue
        s2 = score(q[i], decode_second(take(enc, c), means), metric)[0]
        out_ids[i], out_s[i] = topk(s2, c, k, metric)
    return out_ids, out_s


def _first_level_topk(enc, means, q, ids, k1, metric, chunk):
    """Top-k1 by first-level score of each query over the rows ``ids``.

    The rows are visited in chunks of ``chunk`` rows; the top-k1 of a union
    is the top-k1 of the per-chunk top-k1 lists, so chunking changes nothing
    but memory use."""
    nq = len(q)
    best_ids = [np.empty(0, np.int64) for _ in range(nq)]
    best_s = [np.empty(0, F64) for _ in range(nq)]
    for s in range(0, len(ids), chunk):
        rows = ids[s:s + chunk]
        sc = score(q, decode_first(take(enc, rows), means), metric)
        for i in range(nq):
            all_ids = np.concatenate([best_ids[i], rows])
            all_s = np.concatenate([best_s[i], sc[i]])
            order = best_first(all_s, all_ids, metric)[:k1]
            best_ids[i], best_s[i] = all_ids[order], all_s[order]
    return best_ids, best_s


def search_exhaustive(enc: dict, means, q, k1: int, k: int, metric: str, live=None,
                      chunk: int = 1 << 16):
    """Brute-force LVQ search over all live rows (Sec. 2.2, App. A.2).

    Stage 1 keeps the k1 best rows by first-level score; stage 2 reorders
    them by the two-level score and keeps k.  With k1 == 0 or no second
    level, the k best by first-level score are returned.  Deleted rows are
    never returned (lazy deletes are filtered from the k results, App. A.2).
    Returns (ids int64 [nq, k], scores float64 [nq, k])."""
    q = np.atleast_2d(np.asarray(q, dtype=F32))
    n = len(enc["lower"])
    live = np.ones(n, dtype=bool) if live is None else np.asarray(live, dtype=bool)
    ids = _live_ids(live)
    two_level = bool(enc.get("bits2")) and k1 > 0
    stage1 = k1 if two_level else k
    cand_ids, cand_s = _first_level_topk(enc, means, q, ids, stage1, metric, chunk)
    if not two_level:
        out_ids = np.full((len(q), k), -1, dtype=np.int64)
        out_s = np.full((len(q), k), pad_value(metric), dtype=F64)
        for i in range(len(q)):
            out_ids[i, :len(cand_ids[i])] = cand_ids[i]
            out_s[i, :len(cand_s[i])] = cand_s[i]
        return out_ids, out_s
    padded = np.full((len(q), k1), -1, dtype=np.int64)
    for i in range(len(q)):
        padded[i, :len(cand_ids[i])] = cand_ids[i]
    return rerank(enc, means, q, padded, k, metric, live)


def first_level_candidates(enc: dict, means, q, k1: int, metric: str, live=None, chunk: int = 1 << 16):
    """Stage 1 alone: the k1 best live rows by first-level score (ids, scores)."""
    q = np.atleast_2d(np.asarray(q, dtype=F32))
    n = len(enc["lower"])
    live = np.ones(n, dtype=bool) if live is None else np.asarray(live, dtype=bool)
    ids, s = _first_level_topk(enc, means, q, _live_ids(live), k1, metric, chunk)
    out_ids = np.full((len(q), k1), -1, dtype=np.int64)
    out_s = np.full((len(q), k1), pad_value(metric), dtype=F64)
    for i in range(len(q)):
        out_ids[i, :len(ids[i])] = ids[i]
        out_s[i, :len(s[i])] = s[i]
    return out_ids, out_s


def search_candidates(enc: dict, means, q, cand, k1: int, k: int, metric: str, live=None):
    """ID-gather form: the search restricted to each query's candidate list.

    Stands in for the frontier scoring of greedy graph search (Alg. 1): ids
    that are negative, out of range, repeated or deleted are skipped; the
    remaining ones are scored on the first level, the k1 best are reranked
    on two levels and the k best are returned."""
    q = np.atleast_2d(np.asarray(q, dtype=F32))
    cand = np.atleast_2d(np.asarray(cand, dtype=np.int64))
    n = len(enc["lower"])
    live = np.ones(n, dtype=bool) if live is None else np.asarray(live, dtype=bool)
    two_level = bool(enc.get("bits2")) and k1 > 0
    stage1 = k1 if two_level else k
    firsts = np.full((len(q), stage1), -1, dtype=np.int64)
    first_s = np.full((len(q), stage1), pad_value(metric), dtype=F64)
    for i in range(len(q)):
        c = cand[i]
        c = np.unique(c[(c >= 0) & (c < n)])
        c = c[live[c]]
        if len(c) == 0:
            continue
        s1 = score(q[i], decode_first(take(enc, c), means), metric)[0]
        firsts[i], first_s[i] = topk(s1, c, stage1, metric)
    if not two_level:
        return firsts, first_s
    return rerank(enc, means, q, firsts, k, metric, live)


def ground_truth(enc: dict, means, q, k: int, metric: str, live=None, chunk: int = 1 << 16):
    """Exact k-NN over the decoded vectors: the k best live rows by the
    two-level score (first level when there is no second level)."""
    q = np.atleast_2d(np.asarray(q, dtype=F32))
    n = len(enc["lower"])
    live = np.ones(n, dtype=bool) if live is None else np.asarray(live, dtype=bool)
    ids = _live_ids(live)
    level = 2 if enc.get("bits2") else 1
    best_ids = [np.empty(0, np.int64) for _ in range(len(q))]
    best_s = [np.empty(0, F64) for _ in range(len(q))]
    for s in range(0, len(ids), chunk):
        rows = ids[s:s + chunk]
        sc = score(q, decode(take(enc, rows), means, level), metric)
        for i in range(len(q)):
            all_ids = np.concatenate([best_ids[i], rows])
            all_s = np.concatenate([best_s[i], sc[i]])
            order = best_first(all_s, all_ids, metric)[:k]
            best_ids[i], best_s[i] = all_ids[order], all_s[order]
    out_ids = np.full((len(q), k), -1, dtype=np.int64)
    out_s = np.full((len(q), k), pad_value(metric), dtype=F64)
    for i in range(len(q)):
        out_ids[i, :len(best_ids[i])] = best_ids[i]
        out_s[i, :len(best_s[i])] = best_s[i]
    return out_ids, out_s


def exact_knn(x: np.ndarray, q, k: int, metric: str, chunk: int = 1 << 16):
    """Exact k-NN of the raw (unquantised) float32 vectors x: the k best rows
    by (score, id) with scores in float64 (the k-NN problem of Sec. 2.1, on
    the original data).  Returns (ids int64 [nq, k], scores float64 [nq, k])."""
    x = np.asarray(x, dtype=F32)
    q = np.atleast_2d(np.asarray(q, dtype=F32))
    best_ids = [np.empty(0, np.int64) for _ in range(len(q))]
    best_s = [np.empty(0, F64) for _ in range(len(q))]
    for s in range(0, len(x), chunk):
        rows = np.arange(s, min(len(x), s + chunk), dtype=np.int64)
        sc = score(q, x[s:s + chunk].astype(F64), metric)
        for i in range(len(q)):
            all_ids = np.concatenate([best_ids[i], rows])
            all_s = np.concatenate([best_s[i], sc[i]])
            order = best_first(all_s, all_ids, metric)[:k]
            best_ids[i], best_s[i] = all_ids[order], all_s[order]
    return np.stack(best_ids), np.stack(best_s)


def recall_at_k(found: np.ndarray, truth: np.ndarray, k: int) -> float:
    """k-recall@k = |S cap G| / k averaged over queries (Sec. 2.1)."""
    found = np.atleast_2d(found)[:, :k]
    truth = np.atleast_2d(truth)[:, :k]
    hits = 0
    for s, g in zip(found, truth):
        hits += len(set(s[s >= 0].tolist()) & set(g[g >= 0].tolist()))
    return hits / (k * len(found))


# --------------------------------------------------------------------------
# M-LVQ centre update (Sec. 3.2): re-encoding a centre's vectors
# --------------------------------------------------------------------------

def reconstruct_f32(enc: dict, means) -> np.ndarray:
    """The stored records decoded in float32, each operation rounded:
    y = D*c + l, plus (second level) D2*c2 + l2, then x = mu_m + y.  This is
    the input of a re-encode, so its rounding is fixed step by step."""
    d = enc["codes1"].shape[1]
    means = np.asarray(means, dtype=F32).reshape(-1, d)
    step = enc["step"].astype(F32)[:, None]
    y = ((step * enc["codes1"].astype(F32)).astype(F32) + enc["lower"].astype(F32)[:, None]).astype(F32)
    if enc.get("bits2"):
        lower2, step2 = residual_grid(enc["step"], enc["bits2"], enc.get("grid2", "text"))
        r = ((step2[:, None] * enc["codes2"].astype(F32)).astype(F32) + lower2[:, None]).astype(F32)
        y = (y + r).astype(F32)
    return (means[enc["mean_id"].astype(np.int64)] + y).astype(F32)


def update_mean(enc: dict, means, m: int, new_mean, live=None):
    """Replace centre m by new_mean and re-encode every live record tagged
    with m against it, from its float32 reconstruction; tags stay m and the
    other records are untouched.  Returns (new enc, new means, count)."""
    d = enc["codes1"].shape[1]
    n = len(enc["lower"])
    live = np.ones(n, dtype=bool) if live is None else np.asarray(live, dtype=bool)
    rows = np.nonzero(live & (enc["mean_id"] == m))[0]
    means2 = np.array(np.asarray(means, dtype=F32).reshape(-1, d), copy=True)
    x = reconstruct_f32(take(enc, rows), means2)
    means2[m] = np.asarray(new_mean, dtype=F32)
    e = encode(x, means2, enc["bits1"], enc.get("bits2") or 0, mean_id=np.full(len(rows), m, dtype=np.uint8),
               grid2=enc.get("grid2", "text"))
    out = dict(enc)
    for key in ("codes1", "codes2", "lower", "step"):
        if enc.get(key) is not None:
            arr = np.array(enc[key], copy=True)
            arr[rows] = e[key]
            out[key] = arr
    return out, means2, len(rows)


# --------------------------------------------------------------------------
# Greedy beam search over a graph (Alg. 1), first-level scores
# --------------------------------------------------------------------------

def beam_search(enc: dict, means, q, graph, starts, L: int, k: int, metric: str, live=None, max_expand=None,
                tol=None):
    """Alg. 1 for each query: a search list of at most L nodes ordered by
    (first-level score, id), seeded with ``starts``; repeatedly expand the
    best node not yet expanded (score its out-neighbours not seen before and
    keep the L best of the list) until every listed node is expanded or
    ``max_expand`` expansions were made.  Deleted nodes are never listed.
    Returns the k best listed (ids int64 [nq, k], scores float64 [nq, k],
    padded with -1 / pad_value).

    With ``tol`` given, a third array flags, per query, whether a decision
    of the search rested on two scores a and b with
    |s_a - s_b| <= tol * (scale_a + scale_b), scale = max(|s|, ||q|| ||x^||):
    scores each known only to within tol * scale (a float32 search) may
    order such a pair either way.  The decisions are the node expanded next
    (the best unexpanded node against the next one) and the cut of the list
    to L nodes (its L-th node against the (L+1)-th).  The final choice of
    the k best is not flagged: it is compared with ties allowed."""
    q = np.atleast_2d(np.asarray(q, dtype=F32))
    graph = np.asarray(graph)
    n = len(enc["lower"])
    live = np.ones(n, dtype=bool) if live is None else np.asarray(live, dtype=bool)
    xh = decode_first(enc, means)
    xn = np.linalg.norm(xh, axis=1)
    out_ids = np.full((len(q), k), -1, dtype=np.int64)
    out_s = np.full((len(q), k), pad_value(metric), dtype=F64)
    ambiguous = np.zeros(len(q), dtype=bool)
    key = (lambda s: s) if metric == L2 else (lambda s: -s)
    for i in range(len(q)):
        sc = score(q[i], xh, metric)[0]
        scl = np.maximum(np.abs(sc), float(np.linalg.norm(q[i].astype(F64))) * xn)

        def close(a, b):
            return tol is not None and abs(sc[a] - sc[b]) <= tol * (scl[a] + scl[b])

        seen = set()
        lst = []                      # (key, id)
        for s in starts:
            s = int(s)
            if 0 <= s < n and live[s] and s not in seen:
                seen.add(s)
                lst.append((key(sc[s]), s))
        lst = sorted(lst)
        if len(lst) > L and close(lst[L - 1][1], lst[L][1]):
            ambiguous[i] = True
        lst = lst[:L]
        expanded = set()
        steps = 0
        while max_expand is None or steps < max_expand:
            todo = [v for v in lst if v[1] not in expanded]
            if not todo:
                break
            nxt = todo[0]
            if len(todo) > 1 and close(nxt[1], todo[1][1]):
                ambiguous[i] = True
            expanded.add(nxt[1])
            steps += 1
            for u in graph[nxt[1]]:
                u = int(u)
                if u < 0 or u >= n or u in seen or not live[u]:
                    continue
                seen.add(u)
                lst.append((key(sc[u]), u))
            lst = sorted(lst)
            if len(lst) > L and close(lst[L - 1][1], lst[L][1]):
                ambiguous[i] = True
            lst = lst[:L]
        top = lst[:k]
        out_ids[i, :len(top)] = [u for _, u in top]
        out_s[i, :len(top)] = [sc[u] for _, u in top]
    if tol is not None:
        return out_ids, out_s, ambiguous
    return out_ids, out_s


# --------------------------------------------------------------------------
# Quantisation error (Eq. 5) and its residual-level analogue
# --------------------------------------------------------------------------

def eps_first(x: np.ndarray, means, enc: dict) -> float:
    """Eq. 5: sum_i ||x_i - mu_* - Q(x_i)||^2 with Q(x) = l + D c, float64."""
    x1 = decode_first(enc, means)
    diff = np.asarray(x, dtype=F64) - x1
    return float((diff * diff).sum())


def eps_second(x: np.ndarray, means, enc: dict) -> float:
    """sum_i ||x_i - mu_* - Q(x_i) - Q_res(r_i)||^2, float64."""
    x2 = decode_second(enc, means)
    diff = np.asarray(x, dtype=F64) - x2
    return float((diff * diff).sum())


# --------------------------------------------------------------------------
# The store's slot policy (add / delete with universal ids, Sec. 2.1)
# --------------------------------------------------------------------------

class StoreFull(Exception):
    pass


class SlotReplay:
    """Replays the slot map of the device store.

    An insert of n vectors takes the n lowest-numbered free slots, in
    increasing order, or fails as a whole when fewer are free.  A delete
    frees every listed slot that is live; ids that are out of range, not
    live, or repeated count once at most.  It returns the number freed."""

    def __init__(self, capacity: int):
        self.live = np.zeros(int(capacity), dtype=bool)

    def insert(self, n: int) -> np.ndarray:
        free = np.nonzero(~self.live)[0]
        if len(free) < n:
            raise StoreFull(f"{n} requested, {len(free)} free")
        ids = free[:n].astype(np.int64)
        self.live[ids] = True
        return ids

    def delete(self, ids) -> int:
        ids = np.asarray(ids, dtype=np.int64)
        ids = np.unique(ids[(ids >= 0) & (ids < len(self.live))])
        ids = ids[self.live[ids]]
        self.live[ids] = False
        return int(len(ids))

"""How sensitive LVQ is to the centre it is built with, on synthetic data
(the paper's questions on estimating the mean from a sample and on
distribution shift, Sec. 3 and its experiments, asked of a seeded Gaussian
mixture instead of its datasets).

For a store of mixture vectors it reports, per case, the first-level
quantisation error per vector (Eq. 5 divided by the number of vectors) and
the recall@10 of the two-level search against the exact top-10 of the raw
float32 vectors:

* sample: the centre is the mean of a 1 %, 5 %, 10 % or 100 % sample;
* shift: the store holds vectors of the original components and of new
  ones, all coded with the mean of the original data ("stale"), then the
  centre is moved to the mean of all data with lvq_update_mean
  ("updated": re-encoded from the stored reconstructions) or the vectors
  are inserted afresh with that mean ("fresh").

Encoding, search and the centre update run in the library's kernels; the
error and the ground truth are measurement, computed with torch on the GPU
in float64 (the exact k-NN of the raw vectors, ties to the lower id).
Run: python -m paper_2402_02044_b300.robustness [--n N] [--d D].
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

import synth

from .lvq import Store


def eps1_per_vector(st: Store, x: torch.Tensor, ids: torch.Tensor, means: torch.Tensor) -> float:
    """First-level quantisation error (Eq. 5) divided by the number of vectors:
    mean over rows of ||x - mu_m - (l + D c)||^2 from the stored records,
    summed in float64."""
    e = st.export(ids)
    xh = means[e["mean_id"].long()].double() + e["lower"].double()[:, None] + \
        e["step"].double()[:, None] * e["codes1"].double()
    return float(((x.double() - xh) ** 2).sum(1).mean())


def raw_truth(x: torch.Tensor, q: torch.Tensor, metric: str, k: int = 10) -> torch.Tensor:
    """Ids of the exact k nearest raw vectors of each query, scored in
    float64 and ordered by (score, id)."""
    xd, qd = x.double(), q.double()
    if metric == "ip":
        key = -(qd @ xd.T)
    else:
        key = (qd * qd).sum(1, keepdim=True) - 2 * qd @ xd.T + (xd * xd).sum(1)[None]
    # stable sort: equal scores keep ascending id order
    return torch.sort(key, dim=1, stable=True).indices[:, :k]


def decoded_truth(st: Store, q: torch.Tensor, k: int = 10, level: int = 2, n_rows: int = None,
                  chunk: int = 1 << 20) -> torch.Tensor:
    """Ids of the exact k best live slots of each query by the score of the
    decoded vectors at ``level`` (2: both levels), in float64 and ordered by
    (score, id): the ground truth of recall@k for the store's own search.
    The records are read back with lvq_export and decoded with torch in
    float64 (x^ = mu_m + l + D c [+ l2 + D2 c2]), ``chunk`` slots at a time;
    ``n_rows`` bounds the slots visited (default: the store's capacity)."""
    n = st.capacity if n_rows is None else n_rows
    means = torch.from_numpy(st.means).cuda().double()
    qd = q.double()
    ip = st.metric == "ip"
    best_key = torch.full((len(q), 0), 0.0, dtype=torch.float64, device=q.device)
    best_id = torch.full((len(q), 0), 0, dtype=torch.int64, device=q.device)
    live_bits = st.live_snapshot()
    torch.cuda.synchronize()
    for s in range(0, n, chunk):
        ids = torch.arange(s, min(n, s + chunk), device=q.device)
        w = live_bits[ids >> 5].long() & 0xFFFFFFFF
        alive = ((w >> (ids & 31)) & 1).bool()
        ids = ids[alive]
        if len(ids) == 0:
            continue
        e = st.export(ids)
        x = means[e["mean_id"].long()] + e["lower"].double()[:, None] + e["step"].double()[:, None] * e["codes1"].double()
        if level == 2 and st.bits2:
            step = e["step"]
            lower2 = (-step * 0.5).double()  # exact halving
            step2 = (step / 255.0).double()   # D2 = fl32(D / 255), the residual grid
            x = x + lower2[:, None] + step2[:, None] * e["codes2"].double()
        if ip:
            key = -(qd @ x.T)
        else:
            key = (qd * qd).sum(1, keepdim=True) - 2 * qd @ x.T + (x * x).sum(1)[None]
        kk = min(k + 8, key.shape[1])
        top = torch.topk(key, kk, dim=1, largest=False)
        best_key = torch.cat([best_key, top.values], 1)
        best_id = torch.cat([best_id, ids[top.indices]], 1)
        # keep the k + 8 best so far by (score, id)
        order = torch.argsort(best_id, dim=1, stable=True)
        bk, bi = best_key.gather(1, order), best_id.gather(1, order)
        order = torch.argsort(bk, dim=1, stable=True)[:, :k + 8]
        best_key, best_id = bk.gather(1, order), bi.gather(1, order)
    return best_id[:, :k]


def recall(found: torch.Tensor, truth: torch.Tensor, k: int = 10) -> float:
    """k-recall@k (Sec. 2.1): |found cap truth| / k averaged over queries."""
    hits = sum(len(set(a[a >= 0].tolist()) & set(b.tolist())) for a, b in zip(found[:, :k].cpu(), truth[:, :k].cpu()))
    return hits / (float(k) * len(found))


def _recall(st: Store, x: torch.Tensor, q: torch.Tensor, metric: str, k1: int) -> float:
    got, _ = st.search(q, 10, k1, "auto")
    return recall(got, raw_truth(x, q, metric, 10), 10)


def _eps1(st: Store, x: torch.Tensor, ids: torch.Tensor, means: torch.Tensor) -> float:
    return eps1_per_vector(st, x, ids, means)


def run(n: int = 200_000, d: int = 96, nq: int = 500, metric: str = "l2", fractions=(0.01, 0.05, 0.1, 1.0),
        bits1: int = 4, bits2: int = 8, k1: int = 100, seed: int = 2024) -> list:
    rows = []
    old_c, new_c = 32, 8
    mix = synth.Mixture(d=d, n_comp=old_c + new_c, sigma=0.3, normalize=metric == "ip", seed=seed)
    x_np = mix.rows(0, n, comps=np.arange(old_c))
    q = torch.from_numpy(mix.queries(nq, comps=np.arange(old_c))).cuda()
    x = torch.from_numpy(x_np).cuda()
    ids = torch.arange(n, device="cuda")
    g = np.random.default_rng(seed)
    for f in fractions:
        sample = x_np[np.sort(g.choice(n, max(1, int(f * n)), replace=False))]
        mu = synth.sample_mean(sample)[None]
        st = Store(d, bits1, bits2, mu, metric, n)
        st.insert(x)
        rows.append({"case": f"sample {100 * f:g}%", "eps1_per_vector": _eps1(st, x, ids, torch.from_numpy(mu).cuda()),
                     "recall_at_10": _recall(st, x, q, metric, k1)})
        st.close()
    # shift: half the store from new components, coded with the old mean
    half = n // 2
    x_old = x_np[:half]
    x_new = mix.rows(0, n - half, stream=17, comps=np.arange(old_c, old_c + new_c))
    xs_np = np.concatenate([x_old, x_new])
    xs = torch.from_numpy(xs_np).cuda()
    qs = torch.from_numpy(mix.rows(0, nq, stream=19)).cuda()
    mu_old = synth.sample_mean(x_old)[None]
    mu_all = synth.sample_mean(xs_np)[None]
    st = Store(d, bits1, bits2, mu_old, metric, n)
    st.insert(xs)
    new_ids = torch.arange(half, n, device="cuda")
    rows.append({"case": "shift: stale centre", "eps1_per_vector": _eps1(st, xs, ids, torch.from_numpy(mu_old).cuda()),
                 "eps1_new_vectors": _eps1(st, xs[half:], new_ids, torch.from_numpy(mu_old).cuda()),
                 "recall_at_10": _recall(st, xs, qs, metric, k1)})
    st.update_mean(0, torch.from_numpy(mu_all[0]).cuda())
    rows.append({"case": "shift: centre updated (re-encoded from the store)",
                 "eps1_per_vector": _eps1(st, xs, ids, torch.from_numpy(mu_all).cuda()),
                 "eps1_new_vectors": _eps1(st, xs[half:], new_ids, torch.from_numpy(mu_all).cuda()),
                 "recall_at_10": _recall(st, xs, qs, metric, k1)})
    st.close()
    st = Store(d, bits1, bits2, mu_all, metric, n)
    st.insert(xs)
    rows.append({"case": "shift: fresh encode with the new centre",
                 "eps1_per_vector": _eps1(st, xs, ids, torch.from_numpy(mu_all).cuda()),
                 "eps1_new_vectors": _eps1(st, xs[half:], new_ids, torch.from_numpy(mu_all).cuda()),
                 "recall_at_10": _recall(st, xs, qs, metric, k1)})
    st.close()
    return rows


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--n", type=int, default=200_000)
    ap.add_argument("--d", type=int, default=96)
    ap.add_argument("--nq", type=int, default=500)
    ap.add_argument("--metric", default="l2", choices=["l2", "ip"])
    args = ap.parse_args()
    for r in run(args.n, args.d, args.nq, args.metric):
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()

"""Parity at the benchmark's full size, in the launch configuration the
benchmark times: a 10M x 768 M-LVQ-4x8 store (16 centres, inner product)
searched with the whole uneven query mix (12,716 queries in one call).
The oracle cannot search 10M rows, so sampled outputs are checked one by
one: for a few queries, every returned id's score is recomputed by the
oracle from the raw vector (regenerated from its index) and the same
centres, and no row of a random sample of 20k rows that is left out of the
first-level top-100 beats its 100th score."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from helpers import TOL_FP16, TOL_FP32, check_no_device_error, scale

pytestmark = pytest.mark.gpu

WORKLOAD = "mlvq4x8-ip-10m-d768"


def _rows(mix, ids):
    return np.stack([mix.rows(int(i), int(i) + 1, threads=1)[0] for i in ids])


def test_full_size_search_on_sampled_outputs():
    import bench
    from paper_2402_02044_b300 import Store
    w = synth.WORKLOADS[WORKLOAD]
    mix = synth.mixture_for(WORKLOAD)
    n, d = w["n"], w["d"]
    means = synth.kmeans_means(mix.rows(0, w["kmeans_sample"], stream=5), w["n_means"], seed=3003, iters=5)
    st = Store(d, 4, 8, means, "ip", n)
    for s in range(0, n, 1 << 20):
        st.insert(torch.from_numpy(mix.rows(s, min(n, s + (1 << 20)))).cuda())
    sizes = bench.query_mix("full", 4003)
    q = mix.queries(int(sizes.sum()))
    qd = torch.from_numpy(q).cuda()
    gi, gs = st.search(qd, 10, 100, "auto")
    fi, fs = st.first_level(qd, 100, "auto")
    gi, gs, fi, fs = (t.cpu().numpy() for t in (gi, gs, fi, fs))
    g = np.random.default_rng(77)
    picks = np.concatenate([[0], g.choice(len(q), 5, replace=False)])   # query 0 is a batch of one
    blocks = g.choice(n // synth.BLOCK, 5, replace=False)
    sample_ids = np.concatenate([np.arange(b * synth.BLOCK, (b + 1) * synth.BLOCK) for b in blocks])
    xs = np.concatenate([mix.rows(b * synth.BLOCK, (b + 1) * synth.BLOCK) for b in blocks])
    enc_s = O.encode(xs, means, 4, 8)
    for i in picks:
        # returned ids: the oracle's two-level and first-level scores of their raw vectors
        for ids, sc, level, tol in ((gi[i], gs[i], 2, TOL_FP32), (fi[i], fs[i], 1, TOL_FP16)):
            enc = O.encode(_rows(mix, ids), means, 4, 8)
            xh = O.decode(enc, means, level)
            ref = O.score(q[i], xh, "ip")[0]
            err = np.abs(sc.astype(np.float64) - ref)
            assert np.all(err <= tol * np.maximum(np.abs(ref), scale(q[i], xh, "ip")[0])), (i, level)
        # the sampled rows outside the first-level top-100 do not beat its 100th score
        xh = O.decode_first(enc_s, means)
        s1 = O.score(q[i], xh, "ip")[0]
        out = ~np.isin(sample_ids, fi[i])
        kth = float(fs[i][-1])
        tol = TOL_FP16 * np.maximum(np.abs(s1), scale(q[i], xh, "ip")[0])
        assert np.all(s1[out] <= kth + tol[out]), i
    check_no_device_error(st)
    st.close()

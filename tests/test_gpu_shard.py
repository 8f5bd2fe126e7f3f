"""Row-sharded search with GPU stores: two stores on one GPU, each holding one
slot range of the database, searched through the C ABI; their lists, offset
by the shard base and merged as ``shard.gather_merge`` merges them across
ranks, are held to the oracle.  The first level must be the whole
database's k1 best; the two-level result must be the oracle's re-rank of
the union of the shards' own first-level candidate sets (each shard
re-ranks its own k1)."""
import numpy as np
import pytest
import torch

import oracle as O
from helpers import TOL_FP32, check_no_device_error, check_rerank, check_sorted, check_topk_ids, gmm_case, lib_store
from paper_2402_02044_b300.shard import merge_topk

N, D, NQ, K, K1, WORLD = 3000, 48, 6, 10, 40, 2


@pytest.mark.gpu
@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_sharded_gpu_stores_merge_to_the_oracle(metric):
    x, q, means = gmm_case(N, D, 8, metric, NQ, seed=77)
    qt = torch.from_numpy(q).cuda()
    first, two = [], []
    for r in range(WORLD):
        base, end = r * N // WORLD, (r + 1) * N // WORLD
        st, ids = lib_store(x[base:end], means, 4, 8, metric)
        # a fresh store's slots are 0 .. n-1 in insert order
        assert ids.cpu().numpy().tolist() == list(range(end - base))
        fi, fs = st.first_level(qt, K1, "fp32")
        gi, gs = st.search(qt, K, K1, "fp32")
        check_no_device_error(st)
        st.close()
        first.append((torch.where(fi >= 0, fi + base, fi).cpu(), fs.cpu()))
        two.append((torch.where(gi >= 0, gi + base, gi).cpu(), gs.cpu()))
    enc = O.encode(x, means, 4, 8)
    fi_all = torch.cat([f[0] for f in first], 1)
    fs_all = torch.cat([f[1] for f in first], 1)
    # first level: the merged lists are the whole database's k1 best
    mi, ms = merge_topk(fi_all, fs_all, K1, metric)
    check_sorted(ms, metric)
    check_topk_ids(q, mi, ms, enc, means, metric, K1, TOL_FP32, level=1)
    # two levels: the k best by two-level score over the union of the
    # shards' candidate sets
    wi, ws = merge_topk(torch.cat([t[0] for t in two], 1), torch.cat([t[1] for t in two], 1), K, metric)
    check_sorted(ws, metric)
    check_rerank(q, wi, ws, enc, means, metric, fi_all.numpy().astype(np.int64), K)

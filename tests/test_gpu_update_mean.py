"""GPU parity of the M-LVQ centre update (lvq_update_mean): after replacing
one centre, the stored records of its live vectors are bit-exact with the
oracle's re-encode from their float32 reconstructions, every other record
is unchanged, and searches use the new centre."""
import numpy as np
import pytest
import torch

import oracle as O
from helpers import TOL_FP32, check_no_device_error, check_two_level, gmm_case, lib_store

pytestmark = pytest.mark.gpu


def _records(st, ids):
    e = st.export(torch.from_numpy(ids).cuda())
    return {k: v.cpu().numpy() for k, v in e.items() if v is not None}


def _full(sub, ids, n):
    """Records of the live ids spread over the whole id space (dead rows zero)."""
    out = dict(sub)
    for key in ("codes1", "codes2", "lower", "step", "mean_id"):
        if sub.get(key) is not None:
            arr = np.zeros((n,) + sub[key].shape[1:], sub[key].dtype)
            arr[ids] = sub[key]
            out[key] = arr
    return out


def _oracle_view(rec, bits1, bits2):
    """The exported records as an oracle encoding (codes one per byte)."""
    return {"codes1": rec["codes1"], "codes2": rec.get("codes2") if bits2 else None, "lower": rec["lower"],
            "step": rec["step"], "mean_id": rec["mean_id"], "bits1": bits1, "bits2": bits2}


@pytest.mark.parametrize("metric,bits1,bits2", [("l2", 4, 8), ("ip", 4, 8), ("l2", 8, 0)])
def test_update_mean_matches_the_oracle(metric, bits1, bits2):
    n, d = 6000, 96
    x, q, means = gmm_case(n, d, 16, metric, 8, seed=70 + bits1 + bits2, n_means=4)
    st, ids = lib_store(x, means, bits1, bits2, metric)
    dead = np.arange(0, n, 11)
    st.delete(torch.from_numpy(dead).cuda())
    live = np.ones(n, bool)
    live[dead] = False
    live_ids = np.nonzero(live)[0]
    before = _records(st, live_ids)
    enc = _oracle_view(before, bits1, bits2)
    m = int(np.bincount(before["mean_id"], minlength=4).argmax())
    new_mu = (means[m] + np.float32(0.03) * np.cos(np.arange(d, dtype=np.float32))).astype(np.float32)
    cnt = st.update_mean(m, torch.from_numpy(new_mu).cuda())
    sub, means2, ref_cnt = O.update_mean(enc, means, m, new_mu)
    assert cnt == ref_cnt > 0
    after = _records(st, live_ids)
    for key in ("codes1", "lower", "step", "mean_id") + (("codes2",) if bits2 else ()):
        assert np.array_equal(after[key], sub[key]), key
    ref = _full(sub, live_ids, n)
    # the searches now decode with the new centre
    qt = torch.from_numpy(q).cuda()
    k1 = 50 if bits2 else 0
    gi, gs = st.search(qt, 10, k1, "fp32")
    if bits2:
        check_two_level(q, gi, gs, st.first_level(qt, k1, "fp32"), ref, means2, metric, k1, 10, TOL_FP32, live=live)
    else:
        from helpers import check_topk_ids
        check_topk_ids(q, gi, gs, ref, means2, metric, 10, TOL_FP32, live=live, level=1)
    check_no_device_error(st)
    st.close()


def test_update_mean_rejects_a_bad_index():
    from paper_2402_02044_b300 import lvq as L
    x, q, means = gmm_case(500, 32, 4, "l2", 1, seed=3, n_means=2)
    st, _ = lib_store(x, means, 4, 8, "l2")
    with pytest.raises(L.LVQError):
        st.update_mean(2, torch.zeros(32, device="cuda"))
    st.close()

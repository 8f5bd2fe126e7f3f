"""lvq_search_exhaustive_static: the small-batch search with its scratch in a
file-scope device array.  Its results must equal lvq_search_exhaustive at
LVQ_INT16 on the same store and queries, call after call, and the calls
after the first must leave the device's free memory unchanged.  Collected
last (file name) so that it also runs after every other GPU test."""
import numpy as np
import pytest
import torch

from helpers import gmm_case, lib_store

pytestmark = pytest.mark.gpu

CASES = [
    # n, d, comps, metric, bits1, bits2, n_means, nq, k1, k
    (20000, 768, 32, "ip", 4, 8, 4, 4, 100, 10),
    (9000, 96, 16, "l2", 4, 8, 1, 1, 50, 10),
    (5000, 200, 16, "l2", 8, 8, 1, 3, 0, 20),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "n%d-d%d-%s-%dx%d-q%d-k1_%d" % (c[0], c[1], c[3], c[4], c[5],
                                                                                    c[7], c[8]))
def test_static_scratch_search_matches_the_allocating_entry_point(case):
    from paper_2402_02044_b300 import lvq as L
    n, d, comps, metric, b1, b2, m, nq, k1, k = case
    x, q, means = gmm_case(n, d, comps, metric, nq, seed=900 + d, n_means=m)
    st, _ = lib_store(x, means, b1, b2, metric)
    qt = torch.from_numpy(q).cuda()
    ref_i, ref_s = st.search(qt, k, k1, "int16")
    out_i = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    out_s = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    # first call on the device: looks up the scratch address
    L.lvq_search_exhaustive_static(st.handle, qt, k1, k, out_i, out_s)
    torch.cuda.synchronize()
    assert torch.equal(out_i, ref_i) and torch.equal(out_s, ref_s)
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        out_i.fill_(-7)
        out_s.fill_(0.0)
        L.lvq_search_exhaustive_static(st.handle, qt, k1, k, out_i, out_s)
        torch.cuda.synchronize()
        assert torch.equal(out_i, ref_i) and torch.equal(out_s, ref_s)
    assert torch.cuda.mem_get_info()[0] == free0
    st.close()


def test_static_scratch_search_rejects_what_it_cannot_hold():
    from paper_2402_02044_b300 import lvq as L
    x, q, means = gmm_case(3000, 96, 8, "l2", 5, seed=44)
    st, _ = lib_store(x, means, 4, 8, "l2")
    qt = torch.from_numpy(q).cuda()
    out_i = torch.empty((5, 10), dtype=torch.int64, device="cuda")
    out_s = torch.empty((5, 10), dtype=torch.float32, device="cuda")
    with pytest.raises(L.LVQError) as e:
        L.lvq_search_exhaustive_static(st.handle, qt, 100, 10, out_i, out_s)
    assert e.value.status == L.LVQ_EINVAL
    assert "1 to 4 queries" in L.lvq_last_error(st.handle)[1]
    # a valid call afterwards still works
    L.lvq_search_exhaustive_static(st.handle, qt[:2], 100, 10, out_i[:2], out_s[:2])
    ref_i, _ = st.search(qt[:2], 10, 100, "int16")
    assert torch.equal(out_i[:2], ref_i)
    st.close()

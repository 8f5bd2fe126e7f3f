"""Failure detection on the GPU without a GPU fault: a pipeline wait of the
tensor-core scan given a limit of one poll runs out, the scan records
LVQ_ETIMEOUT in the store and ends its CTAs (after its own copies and MMAs
in flight have finished), the host reads the status, and the same store then
answers a search correctly with the default limit."""
import numpy as np
import pytest
import torch

import oracle as O
from helpers import TOL_FP16, check_no_device_error, check_two_level, gmm_case, lib_store

pytestmark = pytest.mark.gpu


def test_a_wait_that_runs_out_reports_a_timeout_and_the_store_recovers():
    from paper_2402_02044_b300 import lvq as L
    x, q, means = gmm_case(200_000, 768, 32, "ip", 64, seed=19)
    st, _ = lib_store(x, means, 4, 8, "ip")
    qt = torch.from_numpy(q).cuda()
    check_no_device_error(st)
    st.set_tuning(wait_polls=1)
    assert st.get_tuning()["wait_polls"] == 1
    seen = []
    for _ in range(3):  # one poll per wait: some wait of the pipeline gives up
        st.search(qt, 10, 100, "fp16")
        code, msg = L.lvq_last_error(st.handle)
        seen.append(code)
        if code == L.LVQ_ETIMEOUT:
            break
    assert L.LVQ_ETIMEOUT in seen, seen
    # the device is still usable and the store intact: default limit again
    st.set_tuning()
    check_no_device_error(st)
    enc = O.encode(x, means, 4, 8)
    gi, gs = st.search(qt, 10, 100, "fp16")
    check_two_level(q, gi, gs, st.first_level(qt, 100, "fp16"), enc, means, "ip", 100, 10, TOL_FP16)
    check_no_device_error(st)
    st.close()

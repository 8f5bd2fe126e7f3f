"""The centre-robustness experiment on a small store: every case runs, the
error of a sample mean approaches that of the full mean as the sample
grows, and under shift re-encoding from the stored records with the new
centre costs little more than a fresh encode."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_robustness_cases():
    from paper_2402_02044_b300 import robustness
    rows = robustness.run(n=40_000, d=48, nq=200, fractions=(0.01, 1.0))
    by = {r["case"]: r for r in rows}
    s1, s100 = by["sample 1%"], by["sample 100%"]
    assert np.isfinite(s1["eps1_per_vector"]) and s100["eps1_per_vector"] <= s1["eps1_per_vector"] * 1.05
    assert s100["recall_at_10"] >= 0.5
    stale = by["shift: stale centre"]
    upd = by["shift: centre updated (re-encoded from the store)"]
    fresh = by["shift: fresh encode with the new centre"]
    assert np.isfinite(stale["eps1_new_vectors"]) and upd["recall_at_10"] >= 0.5
    # the stored two-level reconstructions are within a residual step of the
    # vectors, so the re-encode is almost as good as encoding them afresh
    assert upd["eps1_per_vector"] <= fresh["eps1_per_vector"] * 1.05

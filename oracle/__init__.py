"""CPU oracle for LVQ search (arxiv 2402.02044) -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct restatement of what the GPU path computes:
LVQ / M-LVQ encoding (Eq. 1-3, Def. 1), decoding in float64, brute-force
scoring (Sec. 3.2, "Euclidean distance" and "Inner product" paragraphs),
top-k with lazy-delete filtering (App. A.2), residual re-ranking (Sec. 2.2,
App. C), k-recall@k (Sec. 2.1), the first-level quantisation error (Eq. 5) and
a replay of the store's slot policy.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library never calls it, and it
shares no code with the CUDA path; the only common dependency is the seeded
input generator in ``synth``.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(hand-worked values, closed forms, invariants, brute force on small inputs)
except the recall numbers quoted by the paper, whose datasets are absent:
recall is "parity unpinned" against the paper.
"""
from .lvq import *  # noqa: F401,F403

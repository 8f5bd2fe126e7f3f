"""A search graph for lvq_search_graph, built with the library's own scans.

The paper's graph construction (Vamana/FreshVamana) is out of scope; this
builds a stand-in that greedy search can navigate: each node's R_near
nearest neighbours by the store's first-level search (queries = the stored
vectors themselves) plus R_far uniformly drawn long-range edges, which
connect the clusters a pure k-NN graph of a mixture leaves apart.
"""
from __future__ import annotations

import numpy as np
import torch

from .lvq import Store


def knn_graph(store: Store, x: torch.Tensor, r_near: int = 24, r_far: int = 8, batch: int = 4096,
              seed: int = 0) -> torch.Tensor:
    """int32 [n, r_near + r_far] out-neighbour ids of the n vectors x (stored
    in slots 0 .. n-1): the first r_near by first-level score (the node
    itself excluded), then r_far random nodes."""
    n = x.shape[0]
    near = torch.empty((n, r_near), dtype=torch.int32, device=x.device)
    for s in range(0, n, batch):
        e = min(n, s + batch)
        ids, _ = store.first_level(x[s:e].contiguous(), r_near + 1, "auto")
        self_id = torch.arange(s, e, device=x.device)[:, None]
        # drop the node itself (or the last entry when it was not found)
        pos = torch.arange(r_near + 1, device=x.device)[None, :] + (ids == self_id).long() * (r_near + 2)
        order = torch.argsort(pos, dim=1)[:, :r_near]
        near[s:e] = ids.gather(1, order).to(torch.int32)
    g = np.random.default_rng(seed)
    far = torch.from_numpy(g.integers(0, n, (n, r_far)).astype(np.int32)).to(x.device)
    return torch.cat([near, far], dim=1).contiguous()

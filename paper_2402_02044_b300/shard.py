"""Row-sharded search across ranks: each rank holds a slot range of the
database in its own store, searches it, and the per-shard top-k lists are
gathered and merged into the global top-k by (score, id).

The merge is exact for the first level (the global top-k of a union is the
top-k of the per-part top-k lists).  For the two-level search each shard
re-ranks its own k1 first-level candidates, so the merged result is the
top-k by two-level score over the union of the shards' candidate sets.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

L2, IP = "l2", "ip"


def merge_topk(ids: torch.Tensor, scores: torch.Tensor, k: int, metric: str):
    """Best k of each row of (ids, scores) [nq, m], best first, ties by lower
    id; entries with id -1 (padding) go last.  Returns (ids, scores) [nq, k]."""
    ids = ids.to(torch.int64)
    pad = ids < 0
    key = scores.to(torch.float64) if metric == L2 else -scores.to(torch.float64)
    key = torch.where(pad, torch.full_like(key, float("inf")), key)
    big = torch.iinfo(torch.int64).max
    tie = torch.where(pad, torch.full_like(ids, big), ids)
    o1 = torch.sort(tie, dim=1, stable=True).indices
    key1 = torch.gather(key, 1, o1)
    o2 = torch.sort(key1, dim=1, stable=True).indices
    order = torch.gather(o1, 1, o2)[:, :k]
    out_ids = torch.gather(ids, 1, order)
    out_sc = torch.gather(scores, 1, order)
    fill = torch.full_like(out_sc, float("inf") if metric == L2 else float("-inf"))
    out_sc = torch.where(out_ids < 0, fill, out_sc)
    return out_ids, out_sc


def gather_merge(ids: torch.Tensor, scores: torch.Tensor, shard_base: int, k: int, metric: str, group=None):
    """Offset this rank's shard-local ids by shard_base, all-gather every
    rank's lists and merge them (every rank gets the global result)."""
    gids = torch.where(ids >= 0, ids + shard_base, ids)
    world = dist.get_world_size(group)
    all_ids = [torch.empty_like(gids) for _ in range(world)]
    all_sc = [torch.empty_like(scores) for _ in range(world)]
    dist.all_gather(all_ids, gids.contiguous(), group=group)
    dist.all_gather(all_sc, scores.contiguous(), group=group)
    return merge_topk(torch.cat(all_ids, 1), torch.cat(all_sc, 1), k, metric)


def sharded_search(store, q: torch.Tensor, k: int, k1: int, shard_base: int, precision: str = "auto",
                   group=None):
    """lvq_search_exhaustive on this rank's shard, then the gather-merge."""
    ids, sc = store.search(q, k, k1, precision)
    return gather_merge(ids, sc, shard_base, k, store.metric, group)

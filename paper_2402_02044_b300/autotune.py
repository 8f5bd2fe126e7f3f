"""Autotuner for the scan tile shapes.

For each query-batch size bucket it times the tensor-core first-level scan
with every admissible query-tile width (``mma_n``) and persistent-CTA count
(``mma_ctas``), using the library's own per-kernel event timing, and keeps
the fastest.  Results are cached as JSON keyed by GPU name, d, bits, metric
and database-size bucket.
"""
from __future__ import annotations

import json
import os
from typing import Iterable, Optional

import torch

from . import lvq as L

DEFAULT_SIZES = (1, 16, 64, 256, 1024, 4096)


def _key(store: "L.Store", n_rows: int) -> str:
    name = torch.cuda.get_device_name().replace(" ", "_")
    nb = 1
    while nb < n_rows:
        nb <<= 1
    return f"{name}|d{store.d}|b{store.bits1}x{store.bits2}|{store.metric}|n{nb}"


def candidates(nq: int, sm_count: int, widths=(16, 32, 64, 128), ctas_opts=None) -> list:
    out = []
    for n in widths:
        if n > 16 and n > 2 * max(nq, 1):
            continue
        for ctas in (ctas_opts if ctas_opts is not None else (0, sm_count // 2)):
            out.append({"mma_n": n, "mma_ctas": ctas})
    return out


def time_scan(store: "L.Store", q: torch.Tensor, k1: int, tuning: dict, reps: int = 3) -> float:
    """Mean milliseconds of the tensor-core scan kernel for this batch."""
    store.set_tuning(**tuning)
    store.first_level(q, k1, "fp16")
    torch.cuda.synchronize()
    L.lvq_profile_enable(store.handle, True)
    L.lvq_profile_read(store.handle)
    for _ in range(reps):
        store.first_level(q, k1, "fp16")
    prof = L.lvq_profile_read(store.handle)
    L.lvq_profile_enable(store.handle, False)
    ms, launches = prof["scan_mma"]
    return ms / max(launches, 1)


def autotune(store: "L.Store", queries: torch.Tensor, n_rows: int, sizes: Iterable[int] = DEFAULT_SIZES,
             k1: int = 100, reps: int = 3, cache_path: Optional[str] = None, widths=(16, 32, 64, 128),
             ctas_opts=None) -> dict:
    """Best tuning per batch-size bucket: {bucket: {"mma_n": .., "mma_ctas": ..}}."""
    key = _key(store, n_rows)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return {int(b): t for b, t in cache[key].items()}
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    best = {}
    for nq in sizes:
        q = queries[:nq].contiguous()
        timings = []
        for t in candidates(nq, sm, widths, ctas_opts):
            try:
                timings.append((time_scan(store, q, k1, t, reps), t))
            except L.LVQError:
                continue
        timings.sort(key=lambda p: p[0])
        best[nq] = dict(timings[0][1], ms=timings[0][0])
    store.set_tuning()
    if cache_path:
        cache[key] = {str(b): t for b, t in best.items()}
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return best


def tuning_for(best: dict, nq: int) -> dict:
    """The tuning of the smallest tuned bucket that holds nq queries."""
    for b in sorted(best):
        if nq <= b:
            return {k: v for k, v in best[b].items() if k in ("mma_n", "mma_ctas")}
    b = max(best)
    return {k: v for k, v in best[b].items() if k in ("mma_n", "mma_ctas")}

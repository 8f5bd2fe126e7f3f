"""Seeded synthetic inputs for the LVQ search path.

This module is shared by the oracle, the tests and the benchmark.  It draws
random numbers and arranges them into the shapes of the paper's workloads
(Sec. 4.1, Table 1: d = 96 / 768 / 200 class dimensionalities, 10^4 to 2x10^7
vectors, inner product on unit-normalised data and Euclidean distance).  It
holds none of LVQ's arithmetic: no centring, bounds, step, codes, decoding or
scoring.  The public datasets of the paper are absent, so an isotropic
Gaussian mixture stands in for them:

    component centres  m_c ~ N(0, I_d)                   c = 0 .. C-1
    vector i           z_i ~ U{0..C-1},  x_i = m_{z_i} + sigma * eps_i,
                       eps_i ~ N(0, I_d),  optionally x_i <- x_i / ||x_i||

Rows are produced in fixed blocks of ``BLOCK`` rows.  Block b of stream s is
drawn from ``Philox(key=(seed, s, b))``, so any row range can be regenerated
on its own, on any host, in any order, and by several threads at once (numpy
releases the GIL while filling arrays).

Besides rows the module also prepares two inputs that LVQ takes as given:
the centring means (Sec. 2.2: the sample mean; Sec. 3.2: M centres "computed
using k-means", whose initialisation and iteration count the paper does not
state) and the candidate-ID lists that stand in for a graph-search frontier.
"""
from __future__ import annotations

import concurrent.futures as _cf
import os
from dataclasses import dataclass

import numpy as np

BLOCK = 4096

# stream tags (second word of the Philox key)
_S_CENTRES = 1
_S_BASE = 2
_S_QUERY = 3
_S_CAND = 4
_S_SAMPLE = 5
_S_KMEANS = 6
_S_STREAM = 7
_S_MISC = 8


def _rng(seed: int, stream: int, block: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed), (int(stream) << 32) | int(block)]))


@dataclass(frozen=True)
class Mixture:
    """Isotropic Gaussian mixture with ``n_comp`` components in ``d`` dims."""

    d: int
    n_comp: int
    sigma: float = 0.3
    normalize: bool = False
    seed: int = 0

    def centres(self) -> np.ndarray:
        g = _rng(self.seed, _S_CENTRES)
        return g.standard_normal((self.n_comp, self.d), dtype=np.float32)

    def _block(self, stream: int, b: int, comps: np.ndarray | None, centres: np.ndarray):
        g = _rng(self.seed, stream, b)
        if comps is None:
            z = g.integers(0, self.n_comp, BLOCK, dtype=np.int64)
        else:
            z = comps[g.integers(0, len(comps), BLOCK, dtype=np.int64)]
        eps = g.standard_normal((BLOCK, self.d), dtype=np.float32)
        x = centres[z] + np.float32(self.sigma) * eps
        if self.normalize:
            nrm = np.sqrt(np.einsum("ij,ij->i", x.astype(np.float64), x.astype(np.float64)))
            nrm[nrm == 0] = 1.0
            x = (x / nrm[:, None]).astype(np.float32)
        return x.astype(np.float32, copy=False), z

    def rows(self, start: int, stop: int, *, stream: int = _S_BASE, comps=None,
             threads: int | None = None, with_labels: bool = False):
        """Rows [start, stop) of stream ``stream`` (float32, C-contiguous).

        ``comps`` restricts the draw to a subset of component indices (used
        for the distribution-shift stream, whose inserts come from components
        the initial fill never used)."""
        start, stop = int(start), int(stop)
        n = max(stop - start, 0)
        out = np.empty((n, self.d), dtype=np.float32)
        lab = np.empty(n, dtype=np.int64)
        if n == 0:
            return (out, lab) if with_labels else out
        centres = self.centres()
        comps_a = None if comps is None else np.asarray(comps, dtype=np.int64)
        b0, b1 = start // BLOCK, (stop - 1) // BLOCK

        def fill(b):
            x, z = self._block(stream, b, comps_a, centres)
            lo, hi = max(start, b * BLOCK), min(stop, (b + 1) * BLOCK)
            out[lo - start:hi - start] = x[lo - b * BLOCK:hi - b * BLOCK]
            lab[lo - start:hi - start] = z[lo - b * BLOCK:hi - b * BLOCK]

        nthr = threads if threads is not None else min(32, os.cpu_count() or 1)
        blocks = range(b0, b1 + 1)
        if nthr <= 1 or b1 == b0:
            for b in blocks:
                fill(b)
        else:
            with _cf.ThreadPoolExecutor(nthr) as ex:
                list(ex.map(fill, blocks))
        return (out, lab) if with_labels else out

    def base(self, n: int, **kw):
        return self.rows(0, n, stream=_S_BASE, **kw)

    def queries(self, nq: int, **kw):
        """Held-out queries from the same mixture (a separate stream)."""
        return self.rows(0, nq, stream=_S_QUERY, **kw)

    def labels(self, start: int, stop: int, *, stream: int = _S_BASE, comps=None):
        """Component labels only (cheap: no normals are drawn)."""
        start, stop = int(start), int(stop)
        lab = np.empty(max(stop - start, 0), dtype=np.int64)
        if stop <= start:
            return lab
        comps_a = None if comps is None else np.asarray(comps, dtype=np.int64)
        for b in range(start // BLOCK, (stop - 1) // BLOCK + 1):
            g = _rng(self.seed, stream, b)
            if comps_a is None:
                z = g.integers(0, self.n_comp, BLOCK, dtype=np.int64)
            else:
                z = comps_a[g.integers(0, len(comps_a), BLOCK, dtype=np.int64)]
            lo, hi = max(start, b * BLOCK), min(stop, (b + 1) * BLOCK)
            lab[lo - start:hi - start] = z[lo - b * BLOCK:hi - b * BLOCK]
        return lab


def unit_normal(n: int, d: int, seed: int) -> np.ndarray:
    """n x d standard-normal float32 rows (the Table 3 micro-benchmark setup)."""
    return _rng(seed, _S_MISC).standard_normal((n, d), dtype=np.float32)


def sample_mean(x: np.ndarray) -> np.ndarray:
    """Sample mean accumulated in float64, rounded to float32 (Sec. 2.2)."""
    return np.asarray(x, dtype=np.float64).mean(axis=0).astype(np.float32)


def running_mean(mix: Mixture, n: int, chunk: int = 1 << 18, stream: int = _S_BASE) -> np.ndarray:
    """Sample mean of rows [0, n) of a stream without holding them all."""
    acc = np.zeros(mix.d, dtype=np.float64)
    for s in range(0, n, chunk):
        acc += mix.rows(s, min(n, s + chunk), stream=stream).astype(np.float64).sum(axis=0)
    return (acc / max(n, 1)).astype(np.float32)


def kmeans_means(x: np.ndarray, m: int, seed: int, iters: int = 25) -> np.ndarray:
    """Lloyd's k-means in float64 on the rows of ``x`` (an input fixture).

    Initial centres are ``m`` distinct rows drawn at random; each iteration
    assigns rows to the nearest centre and replaces each centre by the mean of
    its rows; an emptied cluster is reseeded with the row farthest from its
    current centre.  Returns float32 centres [m, d]."""
    x64 = np.asarray(x, dtype=np.float64)
    g = _rng(seed, _S_KMEANS)
    cen = x64[g.choice(len(x64), size=m, replace=False)].copy()
    xx = np.einsum("ij,ij->i", x64, x64)
    for _ in range(iters):
        d2 = xx[:, None] - 2.0 * (x64 @ cen.T) + np.einsum("ij,ij->i", cen, cen)[None, :]
        lab = np.argmin(d2, axis=1)
        for c in range(m):
            sel = lab == c
            if sel.any():
                cen[c] = x64[sel].mean(axis=0)
            else:
                far = int(np.argmax(d2[np.arange(len(x64)), lab]))
                cen[c] = x64[far]
    return cen.astype(np.float32)


def candidate_lists(labels_db: np.ndarray, query_labels: np.ndarray, n_cand: int,
                    frac_own: float, seed: int) -> np.ndarray:
    """Per query, ``n_cand`` distinct database ids: ``round(frac_own*n_cand)``
    drawn without replacement from the query's own mixture component, the
    rest uniformly from the whole database (a graph-search frontier stand-in).
    Returns int64 [nq, n_cand]."""
    n = len(labels_db)
    order = np.argsort(labels_db, kind="stable")
    counts = np.bincount(labels_db, minlength=int(labels_db.max()) + 1)
    offs = np.concatenate([[0], np.cumsum(counts)])
    n_own = int(round(frac_own * n_cand))
    out = np.empty((len(query_labels), n_cand), dtype=np.int64)
    for qi, c in enumerate(query_labels):
        g = _rng(seed, _S_CAND, qi)
        members = order[offs[c]:offs[c + 1]]
        k_own = min(n_own, len(members))
        own = members[g.choice(len(members), size=k_own, replace=False)] if k_own else np.empty(0, np.int64)
        need = n_cand - k_own
        chosen = set(own.tolist())
        rest = []
        while len(rest) < need:
            for v in g.integers(0, n, 2 * (need - len(rest)) + 8).tolist():
                if v not in chosen:
                    chosen.add(v)
                    rest.append(v)
                    if len(rest) == need:
                        break
        row = np.concatenate([own, np.asarray(rest, dtype=np.int64)])
        out[qi] = row[g.permutation(n_cand)]
    return out


def choose(n_pool: int, k: int, seed: int, tag: int = 0) -> np.ndarray:
    """k distinct indices from range(n_pool), seeded (stream ops, samples)."""
    g = _rng(seed, _S_STREAM, tag)
    return np.sort(g.choice(n_pool, size=k, replace=False)).astype(np.int64)


def log_uniform_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """``count`` integers log-uniform in [lo, hi] (uneven query-batch sizes)."""
    g = _rng(seed, _S_MISC, 1)
    v = np.exp(g.uniform(np.log(lo), np.log(hi + 1), count))
    return np.clip(np.floor(v).astype(np.int64), lo, hi)


def poisson_arrivals(count: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process with the given rate."""
    g = _rng(seed, _S_MISC, 2)
    return np.cumsum(g.exponential(1.0 / rate_per_s, count))


def uniform_ints(count: int, lo: int, hi: int, seed: int, tag: int = 3) -> np.ndarray:
    g = _rng(seed, _S_MISC, tag)
    return g.integers(lo, hi + 1, count, dtype=np.int64)


# The workloads of the benchmark and the parity tests (sizes, mixture shape,
# metric).  Seeds: data 1000+i, queries drawn from the same seed's query
# stream.  sigma = 0.3 throughout; inner-product data is unit-normalised.
WORKLOADS = {
    "lvq8-l2-10k-d96": dict(n=10_000, d=96, comps=32, normalize=False, metric="l2", bits1=8, bits2=0,
                            n_means=1, nq=100, k=10, seed=1001),
    "lvq4x8-ip-1m-d768": dict(n=1_000_000, d=768, comps=64, normalize=True, metric="ip", bits1=4,
                              bits2=8, n_means=1, k1=100, k=10, seed=1002),
    "mlvq4x8-ip-10m-d768": dict(n=10_000_000, d=768, comps=256, normalize=True, metric="ip", bits1=4,
                                bits2=8, n_means=16, kmeans_sample=100_000, k1=100, k=10, seed=1003),
    "gather-lvq4x8-l2-5m-d96": dict(n=5_000_000, d=96, comps=128, normalize=False, metric="l2", bits1=4,
                                    bits2=8, n_means=1, nq=8192, n_cand=2048, frac_own=0.7, k1=50, k=10,
                                    seed=1004),
    "stream-lvq4x8-l2-20m-d200": dict(n=20_000_000, d=200, comps=128, new_comps=8, normalize=False,
                                      metric="l2", bits1=4, bits2=8, n_means=1, step_frac=0.01, seed=1005),
}


def mixture_for(name: str) -> Mixture:
    w = WORKLOADS[name]
    total = w["comps"] + w.get("new_comps", 0)
    return Mixture(d=w["d"], n_comp=total, sigma=0.3, normalize=w["normalize"], seed=w["seed"])

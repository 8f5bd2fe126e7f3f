"""Continuous-batching serving loop over a device-resident LVQ store.

Host-side scheduling only: every search, insert, delete and publication
runs in liblvq's kernels through the C ABI.

Model
-----
* Query requests (a [b, d] batch and a k) from many clients are concatenated
  into one exhaustive search (one persistent scan launch over uneven request
  sizes) and run on one of several *lanes*: a store view (own scratch
  memory) with its own CUDA stream, so batches overlap on the device.  A
  request's rows are re-split from the batch's results (the top-k of a query
  is the first k of its top-k_max list).  A request of more than max_batch
  rows is cut into parts of at most max_batch rows; once its first part has
  run, lanes alternate between its remaining parts and new requests, so a
  large request does not hold up small ones behind it.  Its future completes
  when the last part does.
* Insert requests are encoded at once on an update stream with
  ``lvq_insert_deferred``: their slots are written while searches run, but
  stay invisible.  Deletes are queued.
* Visibility changes at *epoch* boundaries, without stopping the queries:
  each epoch has a device copy of the visibility bitmap (two, used in turn),
  and a batch searches through its lane's view on its epoch's copy.  At a
  boundary the update stream publishes the pending inserts, deletes with
  ``lvq_delete_hold`` (the slots stay reserved, so no insert overwrites a
  vector an older snapshot still shows), copies the bitmap for the new
  epoch, and frees the slots held at the previous boundary; before it
  rewrites a bitmap or frees slots it waits, on the device, for the batches
  of the epoch before the current one.  New batches wait on the boundary's
  event.  All parts of a request run on the bitmap of the epoch its first
  part ran in (kept for one more epoch; a second boundary waits until such
  a request has launched its last part).  Every query therefore sees exactly
  the store state of the epoch it ran in, and a request's result is the same
  whether it ran alone, split or batched with others.  A deleted slot becomes
  free for inserts one boundary later.
* Admission: each request holds device bytes (its inputs and outputs) while
  in flight; a request waits while the total would exceed the HBM budget,
  and one that could never fit is rejected.
* Optional CUDA graphs: per lane, per power-of-two batch size and per
  visibility bitmap (a graph keeps the bitmap it was captured with), the
  search of a padded batch is captured once and replayed.
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field
from typing import Optional

import numpy as np
import torch

from .lvq import Store

QUERY, INSERT, DELETE = "query", "insert", "delete"


@dataclass
class Request:
    kind: str
    data: np.ndarray
    k: int = 0
    future: Future = field(default_factory=Future)
    t_submit: float = 0.0
    nbytes: int = 0
    epoch: int = -1
    group: Optional["_Group"] = None  # the request this one is a part of
    part: int = 0
    t_launch: float = 0.0  # host time its (first) batch was launched
    lane: int = -1
    pinned: Optional[torch.Tensor] = None  # update rows / ids in page-locked memory (pinned by the client)


class _Group:
    """A query request cut into parts: results are gathered in part order."""

    def __init__(self, parts: int, future: Future, rows: int):
        self.results = [None] * parts
        self.remaining = parts
        self.rest = collections.deque()  # parts not yet queued: they follow the first
        self.future = future
        self.rows = rows
        self.epoch = -1
        self.t_launch = 0.0


def request_bytes(kind: str, n: int, d: int, k: int) -> int:
    """Device bytes a request holds while in flight."""
    if kind == QUERY:
        return n * (4 * d + 12 * k)
    if kind == INSERT:
        return n * (4 * d + 8)
    return n * 8 + 8


class Admission:
    """Byte budget for work in flight (pure host logic)."""

    def __init__(self, budget: int):
        self.budget = int(budget)
        self.used = 0

    def fits_ever(self, nbytes: int) -> bool:
        return nbytes <= self.budget

    def try_take(self, nbytes: int) -> bool:
        if self.used + nbytes > self.budget:
            return False
        self.used += nbytes
        return True

    def give(self, nbytes: int):
        self.used -= nbytes
        assert self.used >= 0


def form_batch(pending: "collections.deque[Request]", max_batch: int, admission: Admission, accept=None):
    """Take query requests from the head of the queue, in order, while the
    batch stays within max_batch rows and the admission budget (and, when
    given, while accept(request) holds)."""
    batch, rows = [], 0
    while pending:
        r = pending[0]
        if accept is not None and not accept(r):
            break
        n = r.data.shape[0]
        if batch and rows + n > max_batch:
            break
        if not admission.try_take(r.nbytes):
            break
        pending.popleft()
        batch.append(r)
        rows += n
        if rows >= max_batch:
            break
    return batch


def bucket(n: int) -> int:
    b = 1
    while b < n:
        b <<= 1
    return b


class LatencyStats:
    def __init__(self):
        self.lat = []
        self.rows = 0
        self.t0 = None
        self.t1 = None
        self.trace = []  # (t_submit, t_launch, t_done, rows, lane, epoch) per request

    def add(self, t_submit: float, t_done: float, rows: int, t_launch: float = 0.0, lane: int = -1,
            epoch: int = -1):
        self.lat.append(t_done - t_submit)
        self.rows += rows
        self.t0 = t_submit if self.t0 is None else min(self.t0, t_submit)
        self.t1 = t_done if self.t1 is None else max(self.t1, t_done)
        self.trace.append((t_submit, t_launch, t_done, rows, lane, epoch))

    def slowest(self, n: int = 5) -> list:
        """The n slowest requests: latency split into the wait before their
        (first) batch was launched and the time from launch to completion."""
        out = []
        for ts, tl, td, rows, lane, ep in sorted(self.trace, key=lambda r: r[0] - r[2])[:n]:
            out.append({"ms": (td - ts) * 1e3, "wait_ms": (tl - ts) * 1e3 if tl else None,
                        "run_ms": (td - tl) * 1e3 if tl else None, "rows": rows, "lane": lane,
                        "at_s": ts - self.t0, "epoch": ep})
        return out

    def summary(self) -> dict:
        if not self.lat:
            return {"requests": 0}
        a = np.asarray(self.lat) * 1e3
        span = max(self.t1 - self.t0, 1e-9)
        return {"requests": len(a), "p50_ms": float(np.percentile(a, 50)), "p99_ms": float(np.percentile(a, 99)),
                "mean_ms": float(a.mean()), "qps": self.rows / span}


class _Lane:
    def __init__(self, store: Store, d: int, max_batch: int, kmax: int, k1: int):
        self.view = store.view()
        self.view.reserve(max_batch, max(k1, kmax))
        self.stream = torch.cuda.Stream()
        self.q_pin = torch.empty((max_batch, d), dtype=torch.float32).pin_memory()
        self.q_dev = torch.zeros((max_batch, d), dtype=torch.float32, device="cuda")
        self.ids_dev = torch.empty((max_batch, kmax), dtype=torch.int64, device="cuda")
        self.sc_dev = torch.empty((max_batch, kmax), dtype=torch.float32, device="cuda")
        self.ids_pin = torch.empty((max_batch, kmax), dtype=torch.int64).pin_memory()
        self.sc_pin = torch.empty((max_batch, kmax), dtype=torch.float32).pin_memory()
        self.graphs = {}
        self.busy = None  # (event, batch, rows, kb)
        self.busy_epoch = -1


class Server:
    def __init__(self, store: Store, lanes: int = 2, max_batch: int = 4096, k1: int = 100, kmax: int = 100,
                 precision: str = "auto", hbm_budget: Optional[int] = None, use_graphs: bool = False,
                 tuning: Optional[dict] = None, warmup: bool = True):
        self.store = store
        self.d = store.d
        self.k1 = k1 if store.bits2 else 0
        self.kmax = kmax
        self.max_batch = max_batch
        self.precision = precision
        self.use_graphs = use_graphs
        self.tuning = tuning or {}
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info()
            hbm_budget = free // 2
        self.admission = Admission(hbm_budget)
        self.lanes = [_Lane(store, self.d, max_batch, kmax, max(self.k1, kmax)) for _ in range(lanes)]
        self.upd_stream = torch.cuda.Stream()
        # the visibility bitmaps of the current and the previous epoch
        self.snaps = [store.live_snapshot(stream=self.upd_stream)]
        self.snaps.append(torch.empty_like(self.snaps[0]))
        self.upd_stream.synchronize()
        for lane in self.lanes:
            lane.view.set_live(self.snaps[0])
        self.held = collections.deque()  # (epoch entered, ids) of deletes whose slots are held
        if warmup:
            self._warmup()
        self.pending_q = collections.deque()
        self.pending_upd = collections.deque()
        self.staged = []          # (ids_dev, request) of deferred inserts awaiting publication
        self.deletes = []         # delete requests awaiting the epoch boundary
        self.inflight_upd = []    # (event, request, result tensor, kind)
        self.epoch = 0
        self.epoch_base = 0
        self.epoch_event = None
        self.open_groups = collections.deque()  # split requests with parts still to launch
        self.epoch_events = {}  # epoch -> event of the boundary that opened it (last two)
        self._parts_turn = False
        self.stats = LatencyStats()
        self.rejected = 0
        self._lock = threading.Lock()
        self._wake = threading.Condition(self._lock)
        self._stop = False
        self._thread = threading.Thread(target=self._run, name="lvq-serve", daemon=True)
        self._thread.start()

    def _warmup(self):
        """One search per lane at each batch size that selects a different
        kernel (integer scan for 1, 2 and 3-4 queries; tensor-core tiles of
        16, 32, 64 and 128 queries; the merge for fewer or more queries than
        SMs), so that first-use costs (module loading, kernel attributes,
        scratch) are paid before the first request rather than by it."""
        for lane in self.lanes:
            for nb in (1, 2, 4, 16, 32, 64, 128, 256):
                if nb <= self.max_batch:
                    with torch.cuda.stream(lane.stream):
                        self._search(lane, nb, self.kmax)
            lane.stream.synchronize()

    # ------------------------------------------------------------ client API
    def submit_query(self, q: np.ndarray, k: int) -> Future:
        q = np.ascontiguousarray(q, dtype=np.float32).reshape(-1, self.d)
        if not 1 <= k <= self.kmax or q.shape[0] < 1:
            raise ValueError("k or batch size out of range")
        if q.shape[0] <= self.max_batch:
            return self._submit(Request(QUERY, q, k, nbytes=request_bytes(QUERY, len(q), self.d, k)))
        fut = Future()
        cuts = list(range(0, q.shape[0], self.max_batch))
        grp = _Group(len(cuts), fut, q.shape[0])
        t = time.perf_counter()
        parts = [Request(QUERY, q[a:a + self.max_batch], k, t_submit=t, group=grp, part=i,
                         nbytes=request_bytes(QUERY, len(q[a:a + self.max_batch]), self.d, k))
                 for i, a in enumerate(cuts)]
        with self._lock:
            if any(not self.admission.fits_ever(r.nbytes) for r in parts):
                self.rejected += 1
                fut.set_exception(MemoryError("request larger than the HBM budget"))
                return fut
            grp.rest.extend(parts[1:])
            self.pending_q.append(parts[0])
            self._wake.notify_all()
        return fut

    def submit_insert(self, x: np.ndarray) -> Future:
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, self.d)
        # page-locked on the caller's thread, so that the scheduler's copy to
        # the device neither blocks it nor allocates pinned memory there
        return self._submit(Request(INSERT, x, nbytes=request_bytes(INSERT, len(x), self.d, 0),
                                    pinned=torch.from_numpy(x).pin_memory()))

    def submit_delete(self, ids: np.ndarray) -> Future:
        ids = np.ascontiguousarray(ids, dtype=np.int64).reshape(-1)
        return self._submit(Request(DELETE, ids, nbytes=request_bytes(DELETE, len(ids), self.d, 0),
                                    pinned=torch.from_numpy(ids).pin_memory()))

    def reset_stats(self):
        """Forget the latencies recorded so far (e.g. after a warm-up)."""
        with self._lock:
            self.stats = LatencyStats()
            self.epoch_base = self.epoch

    def stats_summary(self) -> dict:
        with self._lock:
            s = self.stats.summary()
            s.update(rejected=self.rejected, epochs=self.epoch - self.epoch_base, hbm_budget=self.admission.budget,
                     slowest=self.stats.slowest())
            return s

    def drain(self, timeout: float = 60.0):
        """Wait until every submitted request has completed."""
        t_end = time.time() + timeout
        while time.time() < t_end:
            with self._lock:
                idle = (not self.pending_q and not self.open_groups and not self.pending_upd and not self.staged
                        and not self.deletes and not self.inflight_upd and all(l.busy is None for l in self.lanes))
            if idle:
                return
            time.sleep(0.001)
        raise TimeoutError("serving loop did not drain")

    def close(self):
        with self._lock:
            self._stop = True
            self._wake.notify_all()
        self._thread.join()
        torch.cuda.synchronize()
        with torch.cuda.stream(self.upd_stream):
            while self.held:
                self.store.release(self.held.popleft()[1], stream=self.upd_stream)
        self.upd_stream.synchronize()
        for l in self.lanes:
            l.view.set_live(None)
            l.view.close()

    def _submit(self, r: Request) -> Future:
        r.t_submit = time.perf_counter()
        with self._lock:
            if not self.admission.fits_ever(r.nbytes):
                self.rejected += 1
                r.future.set_exception(MemoryError("request larger than the HBM budget"))
                return r.future
            (self.pending_q if r.kind == QUERY else self.pending_upd).append(r)
            self._wake.notify_all()
        return r.future

    # ------------------------------------------------------------- scheduler
    def _run(self):
        torch.cuda.set_device(self.store_device())
        while True:
            with self._lock:
                if self._stop:
                    return
                if not (self.pending_q or self.open_groups or self.pending_upd or self.staged or self.deletes
                        or self.inflight_upd or any(l.busy is not None for l in self.lanes)):
                    self._wake.wait(timeout=0.01)
                    continue
            progressed = self._step()
            if not progressed:
                time.sleep(0.0002)

    def store_device(self) -> int:
        return torch.cuda.current_device()

    def _step(self) -> bool:
        progressed = self._complete()
        progressed |= self._stage_updates()
        updates_waiting = bool(self.staged or self.deletes)
        # a split request runs on its first part's bitmap, which the next
        # boundary keeps and the one after rewrites
        if updates_waiting and all(g.epoch == self.epoch for g in self.open_groups):
            self._epoch_boundary()
            progressed = True
        progressed |= self._launch_queries()
        return progressed

    def _complete(self) -> bool:
        done_any = False
        for lane in self.lanes:
            if lane.busy is None or not lane.busy[0].query():
                continue
            _, batch, rows, kb = lane.busy
            lane.busy = None
            t = time.perf_counter()
            ids = lane.ids_pin[:rows, :kb].numpy()
            sc = lane.sc_pin[:rows, :kb].numpy()
            off = 0
            with self._lock:
                for r in batch:
                    n = r.data.shape[0]
                    res = (ids[off:off + n, :r.k].copy(), sc[off:off + n, :r.k].copy())
                    off += n
                    self.admission.give(r.nbytes)
                    g = r.group
                    if g is None:
                        r.future.set_result(res + (r.epoch,))
                        self.stats.add(r.t_submit, t, n, r.t_launch, r.lane, r.epoch)
                        continue
                    g.results[r.part] = res
                    g.remaining -= 1
                    if g.remaining == 0:
                        g.future.set_result((np.concatenate([a for a, _ in g.results]),
                                             np.concatenate([b for _, b in g.results]), g.epoch))
                        self.stats.add(r.t_submit, t, g.rows, g.t_launch, r.lane, g.epoch)
            done_any = True
        keep = []
        for item in self.inflight_upd:
            ev, r, res, kind = item
            if not ev.query():
                keep.append(item)
                continue
            with self._lock:
                self.admission.give(r.nbytes)
            r.future.set_result(int(res.item()) if kind == DELETE else res.numpy())
            done_any = True
        self.inflight_upd = keep
        return done_any

    def _stage_updates(self) -> bool:
        with self._lock:
            if not self.pending_upd:
                return False
            reqs = []
            while self.pending_upd and self.admission.try_take(self.pending_upd[0].nbytes):
                reqs.append(self.pending_upd.popleft())
        if not reqs:
            return False
        with torch.cuda.stream(self.upd_stream):
            for r in reqs:
                # the rows (ids) reach the device in stream order, without a
                # host wait: the copy is from memory the client pinned
                dev = torch.empty(r.data.shape, dtype=r.pinned.dtype, device="cuda")
                dev.copy_(r.pinned, non_blocking=True)
                if r.kind == INSERT:
                    ids = self.store.insert_deferred(dev, stream=self.upd_stream)
                    self.staged.append((ids, dev, r))
                else:
                    self.deletes.append((r, dev))
        return True

    def _epoch_boundary(self):
        """Publish staged inserts, apply queued deletes and take the new
        epoch's bitmap, on the update stream, while batches run."""
        s = self.upd_stream
        e = self.epoch
        nxt = self.snaps[(e + 1) & 1]
        with torch.cuda.stream(s):
            # nxt and the slots held at the previous boundary may still be in
            # use by batches of epoch e - 1
            for lane in self.lanes:
                if lane.busy is not None and lane.busy_epoch < e:
                    s.wait_event(lane.busy[0])
            while self.held:
                self.store.release(self.held.popleft()[1], stream=s)
            for ids, x, r in self.staged:
                self.store.publish(ids, stream=s)
                ids_host = torch.empty(ids.shape, dtype=ids.dtype, pin_memory=True)
                ids_host.copy_(ids, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(s)
                self.inflight_upd.append((ev, r, ids_host, INSERT))
            for r, ids in self.deletes:
                out = self.store.delete_hold(ids, stream=s)
                self.held.append((e + 1, ids))
                ev = torch.cuda.Event()
                ev.record(s)
                self.inflight_upd.append((ev, r, out, DELETE))
            self.store.live_snapshot(nxt, stream=s)
            ev = torch.cuda.Event()
            ev.record(s)
        self.staged, self.deletes = [], []
        self.epoch_event = ev
        self.epoch = e + 1
        self.epoch_events[e + 1] = ev
        self.epoch_events.pop(e - 1, None)

    def _launch_queries(self) -> bool:
        """Start a batch on every idle lane: either the next part of the oldest
        open split request (on that request's epoch) or new requests from the
        queue head (on the current epoch), taking turns when both wait."""
        launched = False
        for lane in self.lanes:
            if lane.busy is not None:
                continue
            batch, epoch = [], self.epoch
            with self._lock:
                take_part = bool(self.open_groups) and (self._parts_turn or not self.pending_q)
                if take_part:
                    g = self.open_groups[0]
                    if self.admission.try_take(g.rest[0].nbytes):
                        batch, epoch = [g.rest.popleft()], g.epoch
                        if not g.rest:
                            self.open_groups.popleft()
                if not batch:
                    batch = form_batch(self.pending_q, self.max_batch, self.admission)
                    for r in batch:
                        g = r.group
                        if g is not None and g.rest:
                            g.epoch = epoch
                            self.open_groups.append(g)
                if not batch and not take_part and self.open_groups:
                    g = self.open_groups[0]
                    if self.admission.try_take(g.rest[0].nbytes):
                        batch, epoch = [g.rest.popleft()], g.epoch
                        if not g.rest:
                            self.open_groups.popleft()
                self._parts_turn = not self._parts_turn
            if not batch:
                break
            rows = sum(r.data.shape[0] for r in batch)
            kb = max(r.k for r in batch)
            t_l = time.perf_counter()
            lane_idx = self.lanes.index(lane)
            for r in batch:
                r.epoch = epoch
                r.t_launch = t_l
                r.lane = lane_idx
                if r.group is not None:
                    r.group.epoch = epoch
                    if not r.group.t_launch:
                        r.group.t_launch = t_l
            self._run_batch(lane, batch, rows, kb, epoch)
            launched = True
        return launched

    def _run_batch(self, lane: _Lane, batch, rows: int, kb: int, epoch: int):
        off = 0
        for r in batch:
            n = r.data.shape[0]
            lane.q_pin[off:off + n].copy_(torch.from_numpy(r.data))
            off += n
        s = lane.stream
        par = epoch & 1
        lane.view.set_live(self.snaps[par])
        lane.busy_epoch = epoch
        with torch.cuda.stream(s):
            ev0 = self.epoch_events.get(epoch)
            if ev0 is not None:
                s.wait_event(ev0)
            lane.q_dev[:rows].copy_(lane.q_pin[:rows], non_blocking=True)
            kk = self.kmax if self.use_graphs else kb
            nb = bucket(rows) if self.use_graphs else rows
            if self.use_graphs:
                # a graph holds the bitmap it was captured with: one per bitmap
                g = lane.graphs.get((nb, par))
                if g is None:
                    g = self._capture(lane, nb, par)
                g.replay()
            else:
                self._search(lane, nb, kk)
            lane.ids_pin[:rows, :kk].copy_(lane.ids_dev[:rows, :kk], non_blocking=True)
            lane.sc_pin[:rows, :kk].copy_(lane.sc_dev[:rows, :kk], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        lane.busy = (ev, batch, rows, kk)

    def _search(self, lane: _Lane, nb: int, kk: int):
        from .lvq import lvq_search_exhaustive
        t = self.tuning.get(bucket(nb))
        if t:
            lane.view.set_tuning(**t)
        ids = lane.ids_dev[:nb, :kk]
        sc = lane.sc_dev[:nb, :kk]
        if kk != lane.ids_dev.shape[1]:
            ids = torch.empty((nb, kk), dtype=torch.int64, device="cuda")
            sc = torch.empty((nb, kk), dtype=torch.float32, device="cuda")
        lvq_search_exhaustive(lane.view.handle, lane.q_dev[:nb], self.k1, kk, self.precision, ids, sc,
                              lane.stream)
        if ids.data_ptr() != lane.ids_dev.data_ptr():
            lane.ids_dev[:nb, :kk].copy_(ids)
            lane.sc_dev[:nb, :kk].copy_(sc)

    def _capture(self, lane: _Lane, nb: int, par: int):
        # a warm-up call outside the capture sets kernel attributes and scratch
        self._search(lane, nb, self.kmax)
        lane.stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=lane.stream):
            self._search(lane, nb, self.kmax)
        lane.graphs[(nb, par)] = g
        return g

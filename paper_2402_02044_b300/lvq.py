"""Python binding of the LVQ C ABI (include/lvq.h), via ctypes.

Argument marshalling only: every function below checks the tensors it is
given (device, dtype, contiguity), passes raw device pointers and the current
CUDA stream to the function of the same name in liblvq.so, and turns a
non-zero status into an ``LVQError``.  All computation happens in the
library's CUDA kernels; there is no fallback.  PyTorch provides device memory
and streams.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblvq.so")

LVQ_OK, LVQ_EINVAL, LVQ_ENOMEM, LVQ_EFULL, LVQ_ENOTFOUND, LVQ_ECUDA, LVQ_ETIMEOUT, LVQ_EBUSY = range(8)
LVQ_L2, LVQ_IP = 0, 1
LVQ_FP32, LVQ_FP16_MMA, LVQ_AUTO, LVQ_INT16 = 0, 1, 2, 3

METRICS = {"l2": LVQ_L2, "ip": LVQ_IP}
PRECISIONS = {"fp32": LVQ_FP32, "fp16": LVQ_FP16_MMA, "auto": LVQ_AUTO, "int16": LVQ_INT16}


class lvq_config(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("bits1", ctypes.c_int32), ("bits2", ctypes.c_int32),
                ("n_means", ctypes.c_int32), ("metric", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("capacity", ctypes.c_int64)]


LVQ_FLAG_LISTING_RESIDUAL = 1
GRIDS = {"text": 0, "listing": LVQ_FLAG_LISTING_RESIDUAL}


class lvq_tuning(ctypes.Structure):
    _fields_ = [("mma_n", ctypes.c_int32), ("mma_ctas", ctypes.c_int32), ("fp32_q", ctypes.c_int32),
                ("fp32_splits", ctypes.c_int32), ("wait_polls", ctypes.c_int32)]


class LVQError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


_lib: Optional[ctypes.CDLL] = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_SIGS = {
    "lvq_create": [ctypes.POINTER(lvq_config), _P, ctypes.POINTER(_P)],
    "lvq_destroy": [_P],
    "lvq_encode": [_P, _P, _I64, _P, _P, _P, _P, _P, _P],
    "lvq_insert": [_P, _P, _I64, _P, _P],
    "lvq_insert_deferred": [_P, _P, _I64, _P, _P],
    "lvq_publish": [_P, _P, _I64, _P],
    "lvq_store_view": [_P, ctypes.POINTER(_P)],
    "lvq_delete": [_P, _P, _I64, _P, _P],
    "lvq_delete_hold": [_P, _P, _I64, _P, _P],
    "lvq_release": [_P, _P, _I64, _P],
    "lvq_live_words": [_P, ctypes.POINTER(_I64)],
    "lvq_snapshot_live": [_P, _P, _P],
    "lvq_view_set_live": [_P, _P],
    "lvq_search_exhaustive": [_P, _P, _I64, _I32, _I32, _I32, _P, _P, _P],
    "lvq_search_first_level": [_P, _P, _I64, _I32, _I32, _P, _P, _P],
    "lvq_update_mean": [_P, _I32, _P, ctypes.POINTER(_I64), _P],
    "lvq_search_graph": [_P, _P, _I64, _P, _I64, _I32, _P, _I32, _I32, _I32, _I32, _I32, _P, _P, _P],
    "lvq_search_exhaustive_static": [_P, _P, _I64, _I32, _I32, _P, _P, _P],
    "lvq_search_candidates": [_P, _P, _I64, _P, _I32, _I32, _I32, _P, _P, _P],
    "lvq_rerank": [_P, _P, _I64, _P, _I32, _I32, _P, _P, _P],
    "lvq_export": [_P, _P, _I64, _P, _P, _P, _P, _P, _P],
    "lvq_stats": [_P, ctypes.POINTER(_I64), _P],
    "lvq_reserve": [_P, _I64, _I32, _I32],
    "lvq_set_tuning": [_P, ctypes.POINTER(lvq_tuning)],
    "lvq_get_tuning": [_P, ctypes.POINTER(lvq_tuning)],
    "lvq_last_error": [_P, ctypes.c_char_p, ctypes.c_size_t],
    "lvq_profile_enable": [_P, _I32],
    "lvq_profile_read": [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64), _I32],
}

KERNEL_KINDS = ["prep", "scan_fp32", "scan_mma", "merge", "gather", "rerank", "insert", "delete", "scan_small"]


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblvq.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing; build it with paper_2402_02044_b300.build.build()")
    lib = ctypes.CDLL(path)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.lvq_status_string.argtypes = [ctypes.c_int]
    lib.lvq_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().lvq_status_string(int(status)).decode()


def _check(status: int, where: str):
    if status != LVQ_OK:
        raise LVQError(status, where)


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _ptr(t: Optional[torch.Tensor], dtype, name: str, allow_none: bool = False) -> Optional[int]:
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


# --------------------------------------------------------------------------
# the C ABI, one Python function per entry point
# --------------------------------------------------------------------------

def lvq_create(d: int, bits1: int, bits2: int, means: np.ndarray, metric: str, capacity: int,
               grid2: str = "text") -> int:
    means = np.ascontiguousarray(means, dtype=np.float32).reshape(-1, d)
    cfg = lvq_config(d, bits1, bits2, len(means), METRICS[metric], GRIDS[grid2], capacity)
    out = _P()
    _check(load().lvq_create(ctypes.byref(cfg), means.ctypes.data_as(_P), ctypes.byref(out)), "lvq_create")
    return out.value


def lvq_destroy(store: int):
    _check(load().lvq_destroy(store), "lvq_destroy")


def lvq_encode(store, x, codes1, codes2, lower, step, mean_id, stream=None):
    n = x.shape[0]
    _check(load().lvq_encode(store, _ptr(x, torch.float32, "x"), n, _ptr(codes1, torch.uint8, "codes1"),
                             _ptr(codes2, torch.uint8, "codes2", True), _ptr(lower, torch.float32, "lower"),
                             _ptr(step, torch.float32, "step"), _ptr(mean_id, torch.uint8, "mean_id"),
                             _stream(stream)), "lvq_encode")


def lvq_insert(store, x, out_ids, stream=None):
    _check(load().lvq_insert(store, _ptr(x, torch.float32, "x"), x.shape[0], _ptr(out_ids, torch.int64, "out_ids"),
                             _stream(stream)), "lvq_insert")


def lvq_insert_deferred(store, x, out_ids, stream=None):
    _check(load().lvq_insert_deferred(store, _ptr(x, torch.float32, "x"), x.shape[0],
                                      _ptr(out_ids, torch.int64, "out_ids"), _stream(stream)), "lvq_insert_deferred")


def lvq_publish(store, ids, stream=None):
    _check(load().lvq_publish(store, _ptr(ids, torch.int64, "ids"), ids.numel(), _stream(stream)), "lvq_publish")


def lvq_store_view(store) -> int:
    out = _P()
    _check(load().lvq_store_view(store, ctypes.byref(out)), "lvq_store_view")
    return out.value


def lvq_delete(store, ids, out_n_deleted, stream=None):
    _check(load().lvq_delete(store, _ptr(ids, torch.int64, "ids"), ids.numel(),
                             _ptr(out_n_deleted, torch.int64, "out_n_deleted"), _stream(stream)), "lvq_delete")


def lvq_delete_hold(store, ids, out_n_deleted, stream=None):
    _check(load().lvq_delete_hold(store, _ptr(ids, torch.int64, "ids"), ids.numel(),
                                  _ptr(out_n_deleted, torch.int64, "out_n_deleted"), _stream(stream)),
           "lvq_delete_hold")


def lvq_release(store, ids, stream=None):
    _check(load().lvq_release(store, _ptr(ids, torch.int64, "ids"), ids.numel(), _stream(stream)), "lvq_release")


def lvq_live_words(store) -> int:
    out = _I64()
    _check(load().lvq_live_words(store, ctypes.byref(out)), "lvq_live_words")
    return out.value


def lvq_snapshot_live(store, dst, stream=None):
    _check(load().lvq_snapshot_live(store, _ptr(dst, torch.int32, "dst"), _stream(stream)), "lvq_snapshot_live")


def lvq_view_set_live(view, live):
    _check(load().lvq_view_set_live(view, _ptr(live, torch.int32, "live", allow_none=True)), "lvq_view_set_live")


def lvq_search_exhaustive(store, q, k1, k, precision, out_ids, out_scores, stream=None):
    _check(load().lvq_search_exhaustive(store, _ptr(q, torch.float32, "q"), q.shape[0], k1, k,
                                        PRECISIONS.get(precision, precision), _ptr(out_ids, torch.int64, "out_ids"),
                                        _ptr(out_scores, torch.float32, "out_scores"), _stream(stream)),
           "lvq_search_exhaustive")


def lvq_search_exhaustive_static(store, q, k1, k, out_ids, out_scores, stream=None):
    _check(load().lvq_search_exhaustive_static(store, _ptr(q, torch.float32, "q"), q.shape[0], k1, k,
                                               _ptr(out_ids, torch.int64, "out_ids"),
                                               _ptr(out_scores, torch.float32, "out_scores"), _stream(stream)),
           "lvq_search_exhaustive_static")


def lvq_update_mean(store, m, new_mean, stream=None) -> int:
    n = _I64(0)
    _check(load().lvq_update_mean(store, m, _ptr(new_mean, torch.float32, "new_mean"), ctypes.byref(n),
                                  _stream(stream)), "lvq_update_mean")
    return int(n.value)


def lvq_search_graph(store, q, graph, starts, L, max_expand, k1, k, out_ids, out_scores, stream=None):
    _check(load().lvq_search_graph(store, _ptr(q, torch.float32, "q"), q.shape[0], _ptr(graph, torch.int32, "graph"),
                                   graph.shape[0], graph.shape[1], _ptr(starts, torch.int64, "starts"),
                                   starts.numel(), L, max_expand, k1, k, _ptr(out_ids, torch.int64, "out_ids"),
                                   _ptr(out_scores, torch.float32, "out_scores"), _stream(stream)),
           "lvq_search_graph")


def lvq_search_first_level(store, q, k1, precision, out_ids, out_scores, stream=None):
    _check(load().lvq_search_first_level(store, _ptr(q, torch.float32, "q"), q.shape[0], k1,
                                         PRECISIONS.get(precision, precision), _ptr(out_ids, torch.int64, "out_ids"),
                                         _ptr(out_scores, torch.float32, "out_scores"), _stream(stream)),
           "lvq_search_first_level")


def lvq_search_candidates(store, q, cand, k1, k, out_ids, out_scores, stream=None):
    _check(load().lvq_search_candidates(store, _ptr(q, torch.float32, "q"), q.shape[0],
                                        _ptr(cand, torch.int64, "cand"), cand.shape[1], k1, k,
                                        _ptr(out_ids, torch.int64, "out_ids"),
                                        _ptr(out_scores, torch.float32, "out_scores"), _stream(stream)),
           "lvq_search_candidates")


def lvq_rerank(store, q, ids, k, out_ids, out_scores, stream=None):
    _check(load().lvq_rerank(store, _ptr(q, torch.float32, "q"), q.shape[0], _ptr(ids, torch.int64, "ids"),
                             ids.shape[1], k, _ptr(out_ids, torch.int64, "out_ids"),
                             _ptr(out_scores, torch.float32, "out_scores"), _stream(stream)), "lvq_rerank")


def lvq_export(store, ids, codes1, codes2, lower, step, mean_id, stream=None):
    _check(load().lvq_export(store, _ptr(ids, torch.int64, "ids"), ids.numel(), _ptr(codes1, torch.uint8, "codes1"),
                             _ptr(codes2, torch.uint8, "codes2", True), _ptr(lower, torch.float32, "lower"),
                             _ptr(step, torch.float32, "step"), _ptr(mean_id, torch.uint8, "mean_id"),
                             _stream(stream)), "lvq_export")


def lvq_stats(store, stream=None) -> int:
    live = _I64()
    _check(load().lvq_stats(store, ctypes.byref(live), _stream(stream)), "lvq_stats")
    return live.value


def lvq_reserve(store, max_nq: int, max_k1: int, max_cand: int = 0):
    _check(load().lvq_reserve(store, max_nq, max_k1, max_cand), "lvq_reserve")


def lvq_set_tuning(store, mma_n=0, mma_ctas=0, fp32_q=0, fp32_splits=0, wait_polls=0):
    t = lvq_tuning(mma_n, mma_ctas, fp32_q, fp32_splits, wait_polls)
    _check(load().lvq_set_tuning(store, ctypes.byref(t)), "lvq_set_tuning")


def lvq_get_tuning(store) -> dict:
    t = lvq_tuning()
    _check(load().lvq_get_tuning(store, ctypes.byref(t)), "lvq_get_tuning")
    return dict(mma_n=t.mma_n, mma_ctas=t.mma_ctas, fp32_q=t.fp32_q, fp32_splits=t.fp32_splits,
                wait_polls=t.wait_polls)


def lvq_profile_enable(store, on: bool = True):
    _check(load().lvq_profile_enable(store, 1 if on else 0), "lvq_profile_enable")


def lvq_profile_read(store) -> dict:
    n = len(KERNEL_KINDS)
    ms = (ctypes.c_double * n)()
    cnt = (_I64 * n)()
    _check(load().lvq_profile_read(store, ms, cnt, n), "lvq_profile_read")
    return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_KINDS)}


def lvq_last_error(store) -> tuple[int, str]:
    buf = ctypes.create_string_buffer(512)
    st = load().lvq_last_error(store, buf, 512)
    return st, buf.value.decode()


# --------------------------------------------------------------------------
# convenience wrapper: owns the handle and allocates output tensors
# --------------------------------------------------------------------------

class Store:
    """A device-resident LVQ store (thin wrapper over the C ABI)."""

    def __init__(self, d: int, bits1: int, bits2: int, means: np.ndarray, metric: str, capacity: int,
                 grid2: str = "text"):
        self.d, self.bits1, self.bits2, self.metric, self.capacity = d, bits1, bits2, metric, capacity
        self.grid2 = grid2
        self.means = np.ascontiguousarray(means, dtype=np.float32).reshape(-1, d)
        self.handle = lvq_create(d, bits1, bits2, self.means, metric, capacity, grid2)

    def close(self):
        if self.handle:
            lvq_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self):
        return torch.device("cuda", torch.cuda.current_device())

    def encode(self, x: torch.Tensor, stream=None):
        n = x.shape[0]
        dev = x.device
        c1 = torch.empty((n, self.d), dtype=torch.uint8, device=dev)
        c2 = torch.empty((n, self.d), dtype=torch.uint8, device=dev) if self.bits2 else None
        lo = torch.empty(n, dtype=torch.float32, device=dev)
        st = torch.empty(n, dtype=torch.float32, device=dev)
        mid = torch.empty(n, dtype=torch.uint8, device=dev)
        lvq_encode(self.handle, x, c1, c2, lo, st, mid, stream)
        return dict(codes1=c1, codes2=c2, lower=lo, step=st, mean_id=mid)

    def insert(self, x: torch.Tensor, stream=None) -> torch.Tensor:
        ids = torch.empty(x.shape[0], dtype=torch.int64, device=x.device)
        lvq_insert(self.handle, x, ids, stream)
        return ids

    def insert_deferred(self, x: torch.Tensor, stream=None) -> torch.Tensor:
        ids = torch.empty(x.shape[0], dtype=torch.int64, device=x.device)
        lvq_insert_deferred(self.handle, x, ids, stream)
        return ids

    def publish(self, ids: torch.Tensor, stream=None):
        lvq_publish(self.handle, ids, stream)

    def view(self) -> "Store":
        """A handle sharing this store's data with its own scratch memory."""
        v = Store.__new__(Store)
        v.d, v.bits1, v.bits2, v.metric, v.capacity = self.d, self.bits1, self.bits2, self.metric, self.capacity
        v.grid2 = self.grid2
        v.means = self.means
        v.handle = lvq_store_view(self.handle)
        v._base = self
        return v

    def delete(self, ids: torch.Tensor, stream=None) -> torch.Tensor:
        out = torch.empty(1, dtype=torch.int64, device=ids.device)
        lvq_delete(self.handle, ids, out, stream)
        return out

    def delete_hold(self, ids: torch.Tensor, stream=None) -> torch.Tensor:
        """Delete, keeping the slots from reuse until release()."""
        out = torch.empty(1, dtype=torch.int64, device=ids.device)
        lvq_delete_hold(self.handle, ids, out, stream)
        return out

    def release(self, ids: torch.Tensor, stream=None):
        lvq_release(self.handle, ids, stream)

    def live_snapshot(self, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """A device copy of the visibility bitmap (int32 words), in stream order."""
        if out is None:
            out = torch.empty(lvq_live_words(self.handle), dtype=torch.int32, device="cuda")
        lvq_snapshot_live(self.handle, out, stream)
        return out

    def set_live(self, live: Optional[torch.Tensor]):
        """(views) search on the given visibility bitmap; None: the store's."""
        lvq_view_set_live(self.handle, live)
        self._live_ref = live

    def search(self, q: torch.Tensor, k: int, k1: int = 0, precision="fp32", stream=None):
        ids = torch.empty((q.shape[0], k), dtype=torch.int64, device=q.device)
        sc = torch.empty((q.shape[0], k), dtype=torch.float32, device=q.device)
        lvq_search_exhaustive(self.handle, q, k1, k, precision, ids, sc, stream)
        return ids, sc

    def search_graph(self, q: torch.Tensor, graph: torch.Tensor, starts: torch.Tensor, k: int, k1: int = 0,
                     L: int = 64, max_expand: int = 0, stream=None):
        ids = torch.empty((q.shape[0], k), dtype=torch.int64, device=q.device)
        sc = torch.empty((q.shape[0], k), dtype=torch.float32, device=q.device)
        lvq_search_graph(self.handle, q, graph.contiguous(), starts.contiguous(), L, max_expand, k1, k, ids, sc,
                         stream)
        return ids, sc

    def update_mean(self, m: int, new_mean: torch.Tensor, stream=None) -> int:
        """Replace centre m and re-encode its live vectors; returns their number."""
        return lvq_update_mean(self.handle, m, new_mean.contiguous(), stream)

    def first_level(self, q: torch.Tensor, k1: int, precision="fp32", stream=None):
        ids = torch.empty((q.shape[0], k1), dtype=torch.int64, device=q.device)
        sc = torch.empty((q.shape[0], k1), dtype=torch.float32, device=q.device)
        lvq_search_first_level(self.handle, q, k1, precision, ids, sc, stream)
        return ids, sc

    def search_candidates(self, q: torch.Tensor, cand: torch.Tensor, k: int, k1: int = 0, stream=None):
        ids = torch.empty((q.shape[0], k), dtype=torch.int64, device=q.device)
        sc = torch.empty((q.shape[0], k), dtype=torch.float32, device=q.device)
        lvq_search_candidates(self.handle, q, cand, k1, k, ids, sc, stream)
        return ids, sc

    def rerank(self, q: torch.Tensor, cand: torch.Tensor, k: int, stream=None):
        ids = torch.empty((q.shape[0], k), dtype=torch.int64, device=q.device)
        sc = torch.empty((q.shape[0], k), dtype=torch.float32, device=q.device)
        lvq_rerank(self.handle, q, cand, k, ids, sc, stream)
        return ids, sc

    def export(self, ids: torch.Tensor, stream=None):
        n = ids.numel()
        dev = ids.device
        c1 = torch.empty((n, self.d), dtype=torch.uint8, device=dev)
        c2 = torch.empty((n, self.d), dtype=torch.uint8, device=dev) if self.bits2 else None
        lo = torch.empty(n, dtype=torch.float32, device=dev)
        st = torch.empty(n, dtype=torch.float32, device=dev)
        mid = torch.empty(n, dtype=torch.uint8, device=dev)
        lvq_export(self.handle, ids, c1, c2, lo, st, mid, stream)
        return dict(codes1=c1, codes2=c2, lower=lo, step=st, mean_id=mid)

    def stats(self, stream=None) -> int:
        return lvq_stats(self.handle, stream)

    def reserve(self, max_nq: int, max_k1: int, max_cand: int = 0):
        lvq_reserve(self.handle, max_nq, max_k1, max_cand)

    def set_tuning(self, **kw):
        lvq_set_tuning(self.handle, **kw)

    def get_tuning(self) -> dict:
        return lvq_get_tuning(self.handle)

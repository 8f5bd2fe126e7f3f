"""The C ABI library loads and exports every entry point that include/lvq.h
declares; argument checks that need no GPU reject bad configurations."""
import ctypes
import os
import re

import pytest

from paper_2402_02044_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lvq.h")


@pytest.fixture(scope="module")
def lib():
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lvq_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_abi():
    names = declared_functions()
    for required in ("lvq_create", "lvq_destroy", "lvq_encode", "lvq_insert", "lvq_delete",
                     "lvq_search_exhaustive", "lvq_search_candidates", "lvq_rerank", "lvq_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    lib.lvq_status_string.restype = ctypes.c_char_p
    assert lib.lvq_status_string(0) == b"ok"
    assert lib.lvq_status_string(3) == b"store full"


@pytest.mark.parametrize("field,value", [("d", 0), ("d", 5000), ("bits1", 1), ("bits1", 9), ("bits2", 1),
                                         ("bits2", 9), ("n_means", 0), ("n_means", 257), ("metric", 2),
                                         ("flags", 2), ("capacity", 0), ("capacity", 1 << 31)])
def test_create_rejects_bad_configs_before_touching_the_device(lib, field, value):
    from paper_2402_02044_b300.lvq import lvq_config
    cfg = dict(d=8, bits1=4, bits2=8, n_means=1, metric=0, flags=0, capacity=16)
    cfg[field] = value
    c = lvq_config(**cfg)
    means = (ctypes.c_float * (8 * 300))()
    out = ctypes.c_void_p()
    lib.lvq_create.argtypes = [ctypes.POINTER(lvq_config), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    assert lib.lvq_create(ctypes.byref(c), means, ctypes.byref(out)) == 1  # LVQ_EINVAL
    assert out.value is None


def test_null_arguments_are_rejected(lib):
    lib.lvq_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.lvq_create(None, None, None) == 1
    lib.lvq_destroy.argtypes = [ctypes.c_void_p]
    assert lib.lvq_destroy(None) == 1


def test_snapshot_and_hold_calls_reject_null_handles(lib):
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    lib.lvq_delete_hold.argtypes = [vp, vp, i64, vp, vp]
    assert lib.lvq_delete_hold(None, None, 0, None, None) == 1
    lib.lvq_release.argtypes = [vp, vp, i64, vp]
    assert lib.lvq_release(None, None, 0, None) == 1
    lib.lvq_live_words.argtypes = [vp, vp]
    w = ctypes.c_int64(0)
    assert lib.lvq_live_words(None, ctypes.byref(w)) == 1
    lib.lvq_snapshot_live.argtypes = [vp, vp, vp]
    assert lib.lvq_snapshot_live(None, None, None) == 1
    lib.lvq_view_set_live.argtypes = [vp, vp]
    assert lib.lvq_view_set_live(None, None) == 1

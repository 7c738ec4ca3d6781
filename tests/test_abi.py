"""The C ABI library without a GPU: it loads, exports every function that
include/cfr.h declares, and answers the calls that need no device (shape
table, static error strings, argument checks made before any device work)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cfr.h")
LIB = os.path.join(ROOT, "paper_2605_14277_b300", "libcfr.so")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)   # drop comments
    names = re.findall(r"^\s*(?:int|void|const\s+char\s*\*)\s*\*?\s*(cfr_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2605_14277_b300 import build
        build.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("cfr_load_tree", "cfr_load_batch", "cfr_iterate", "cfr_get_average_strategy",
                 "cfr_exploitability", "cfr_free", "cfr_strerror", "cfr_load_batch_opts",
                 "cfr_exploitability_batch_noalloc"):
        assert want in names
    assert len(names) >= 20


def test_library_exports_every_declared_function(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_calls_that_need_no_device(lib):
    lib.cfr_strerror.restype = ctypes.c_char_p
    assert lib.cfr_strerror(0)
    assert lib.cfr_strerror(-4)
    n = lib.cfr_num_shapes()
    assert n >= 2
    out = (ctypes.c_int32 * 3)()
    for k in range(1, n + 1):
        assert lib.cfr_shape_info(k, out) == 0
        threads, per_sm, buf = out
        assert threads % 32 == 0 and threads >= 128
        assert per_sm >= 1 and buf % 1024 == 0
        # two buffers per CTA fit an SM's shared memory
        assert per_sm * (2 * buf + 8 * 1024) <= 228 * 1024
    assert lib.cfr_shape_info(0, out) == -6
    assert lib.cfr_shape_info(n + 1, out) == -6
    # the shape chosen when none is given: the default for one game of at
    # least 1M nodes, the 256-thread, 3-CTA, 32 KB shape otherwise
    lib.cfr_pick_shape.argtypes = [ctypes.c_int64, ctypes.c_int64]
    d = lib.cfr_default_shape()
    assert lib.cfr_pick_shape(1, 6_000_000) == d
    many = lib.cfr_pick_shape(64, 2_000_000)
    assert lib.cfr_pick_shape(1, 10_000) == many and many != d
    out3 = (ctypes.c_int32 * 3)()
    assert lib.cfr_shape_info(many, out3) == 0 and list(out3) == [256, 3, 32768]
    assert lib.cfr_pick_shape(0, 10) == -6 and lib.cfr_pick_shape(1, 0) == -6


class _Opts(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int32), ("flat", ctypes.c_int32), ("passes", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 5)]


def test_load_rejects_bad_arguments_before_device_work(lib):
    h = ctypes.c_void_p()
    # no games / NULL output
    assert lib.cfr_load_batch(None, 0, None, ctypes.byref(h)) == -6
    assert lib.cfr_load_batch(None, 1, None, None) == -6
    # bad options are refused before the trees are looked at
    bad = _Opts(99, 0)
    assert lib.cfr_load_batch_opts(None, 1, None, ctypes.byref(bad), ctypes.byref(h)) == -6
    bad = _Opts(0, 2)
    assert lib.cfr_load_batch_opts(None, 1, None, ctypes.byref(bad), ctypes.byref(h)) == -6
    bad = _Opts(0, 0, 3)
    assert lib.cfr_load_batch_opts(None, 1, None, ctypes.byref(bad), ctypes.byref(h)) == -6
    bad = _Opts(0, 0)
    bad.reserved[3] = 1
    assert lib.cfr_load_batch_opts(None, 1, None, ctypes.byref(bad), ctypes.byref(h)) == -6

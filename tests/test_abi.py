"""CPU-side checks of the C ABI: the library builds, loads and exports every
entry point include/qs.h declares; invalid arguments are rejected before any
CUDA call (so these run without a GPU)."""

import ctypes
import os
import re

import pytest

from paper_1601_07195_gb300 import qs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^QS_API\s+[\w\s\*]+?\b(qs_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("qs_create", "qs_apply_1q", "qs_apply_ctrl", "qs_prob", "qs_expect", "qs_grad", "qs_run"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = qs.load()
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert missing == []


def test_version_string():
    assert b"sm_103a" in qs.load().qs_version()


def test_invalid_arguments_rejected_without_gpu():
    lib = qs.load()
    h = ctypes.c_void_p()
    assert lib.qs_create(0, qs.QS_C128, None, ctypes.byref(h)) == qs.QS_EINVAL
    assert lib.qs_create(37, qs.QS_C128, None, ctypes.byref(h)) == qs.QS_EINVAL
    assert lib.qs_create(5, 7, None, ctypes.byref(h)) == qs.QS_EDTYPE
    assert lib.qs_wrap(None, 5, qs.QS_C128, None, ctypes.byref(h)) == qs.QS_EINVAL
    assert lib.qs_wrap(ctypes.c_void_p(8), 5, qs.QS_C128, None, ctypes.byref(h)) == qs.QS_EINVAL  # misaligned
    m = (ctypes.c_double * 8)(*([0.0] * 8))
    assert lib.qs_apply_1q(None, 0, m) == qs.QS_EINVAL
    assert lib.qs_norm(None, None) == qs.QS_EINVAL
    assert lib.qs_set_arith(None, 1) == qs.QS_EINVAL
    assert lib.qs_set_lanes(None, 0) == qs.QS_EINVAL
    assert b"NULL" in lib.qs_last_error()
    assert lib.qs_destroy(None) == qs.QS_OK
    h = ctypes.c_void_p()
    assert lib.qs_wrap(ctypes.c_void_p(1 << 20), 6, qs.QS_C64, None, ctypes.byref(h)) == qs.QS_OK
    assert lib.qs_set_lanes(h, 3) == qs.QS_EINVAL and lib.qs_set_lanes(h, -1) == qs.QS_EINVAL
    assert all(lib.qs_set_lanes(h, m) == qs.QS_OK for m in (qs.LANES_OFF, qs.LANES_AUTO, qs.LANES_ON))
    assert lib.qs_destroy(h) == qs.QS_OK


def test_wrapped_handle_validates_qubits_before_launch():
    # qs_wrap only records the pointer; gate validation happens before any launch
    lib = qs.load()
    h = ctypes.c_void_p()
    assert lib.qs_wrap(ctypes.c_void_p(1 << 20), 4, qs.QS_C128, None, ctypes.byref(h)) == qs.QS_OK
    m = (ctypes.c_double * 8)(*([0.0] * 8))
    assert lib.qs_apply_1q(h, 4, m) == qs.QS_EINVAL
    assert lib.qs_apply_ctrl(h, 1, 1, m) == qs.QS_EINVAL
    assert lib.qs_apply_swap(h, 0, 9) == qs.QS_EINVAL
    assert lib.qs_init_basis(h, 16) == qs.QS_EINVAL
    bad = (ctypes.c_double * 8)(float("nan"), 0, 0, 0, 0, 0, 1, 0)
    assert lib.qs_apply_1q(h, 0, bad) == qs.QS_EINVAL
    assert lib.qs_destroy(h) == qs.QS_OK


def test_host_buffer_arguments_without_gpu():
    lib = qs.load()
    p = ctypes.c_void_p()
    assert lib.qs_host_alloc(0, ctypes.byref(p)) == qs.QS_EINVAL
    assert lib.qs_host_alloc(64, None) == qs.QS_EINVAL
    assert lib.qs_host_free(None) == qs.QS_OK
    assert lib.qs_host_free(ctypes.c_void_p(1 << 20)) == qs.QS_EINVAL  # not from qs_host_alloc

"""Host-side checks of the C ABI (no GPU needed)."""

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nullspace.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ns_[A-Za-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name


def test_binding_declares_every_symbol():
    from paper_2407_04634_gb300 import nullspace
    assert sorted(nullspace.SIGNATURES) == declared_functions()


def test_default_opts(lib):
    from paper_2407_04634_gb300 import nullspace
    o = nullspace.default_opts()
    assert o.eps == 1e-3 and o.refine_tol == 1e-10 and o.stop_factor == 2.0 and o.refine == 1


def test_create_rejects_bad_arguments_or_missing_gpu(lib):
    """Host validation runs before any device work; without a GPU a valid matrix gives
    NS_ERR_CUDA (no CPU fallback)."""
    from paper_2407_04634_gb300 import nullspace as ns
    h = ctypes.c_void_p()
    rp = np.array([0, 1, 3], dtype=np.int64)
    ci = np.array([0, 0, 5], dtype=np.int32)  # 5 is out of range for n = 2
    va = np.ones(3)
    P = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    st = lib.ns_create(ctypes.byref(h), 2, 2, P(rp), P(ci), P(va), 0, 0, 1, 0, None)
    assert st == ns.NS_ERR_INVALID_ARG
    rp_bad = np.array([0, 2, 1], dtype=np.int64)
    st = lib.ns_create(ctypes.byref(h), 2, 2, P(rp_bad), P(ci), P(va), 0, 0, 1, 0, None)
    assert st == ns.NS_ERR_INVALID_ARG
    va_nan = np.array([1.0, np.nan, 1.0])
    ci_ok = np.array([0, 0, 1], dtype=np.int32)
    st = lib.ns_create(ctypes.byref(h), 2, 2, P(rp), P(ci_ok), P(va_nan), 0, 0, 1, 0, None)
    assert st == ns.NS_ERR_INVALID_ARG
    st = lib.ns_create(ctypes.byref(h), 3, 2, P(np.array([0, 1, 2, 3], dtype=np.int64)), P(ci_ok), P(va), 0, 0,
                       1, 1, None)
    assert st == ns.NS_ERR_INVALID_ARG  # spd mode needs a square matrix
    va32_nan = np.array([1.0, np.inf, 1.0], dtype=np.float32)
    st = lib.ns_create(ctypes.byref(h), 2, 2, P(rp), P(ci_ok), P(va32_nan), 1, 0, 1, 0, None)
    assert st == ns.NS_ERR_INVALID_ARG  # FP32 values are checked as FP32
    st = lib.ns_create(ctypes.byref(h), 2, 2, P(rp), P(ci_ok), P(va), 2, 0, 1, 0, None)
    assert st == ns.NS_ERR_INVALID_ARG  # the value-type flag is 0 or 1
    import torch
    if not torch.cuda.is_available():
        st = lib.ns_create(ctypes.byref(h), 2, 2, P(rp), P(ci_ok), P(va), 0, 0, 1, 0, None)
        assert st == ns.NS_ERR_CUDA


def test_null_handle_calls(lib):
    from paper_2407_04634_gb300 import nullspace as ns
    N = ctypes.c_int64()
    assert lib.ns_nullity(None, ctypes.byref(N)) == ns.NS_ERR_INVALID_ARG
    assert lib.ns_solve(None, 1, 30, 1e-10, None) == ns.NS_ERR_INVALID_ARG
    assert lib.ns_last_error(None) == b"null handle"
    lib.ns_destroy(None)

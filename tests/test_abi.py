"""The C-ABI library builds for sm_103a, loads, and exports every declared entry point.

No compute call is made here (no GPU is needed).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"STC_API\s+[\w\s\*]+?\b(stc_\w+)\s*\(", src)
    return names


@pytest.fixture(scope="module")
def libstc():
    from paper_1512_00066_b300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = set(declared_functions())
    for required in ["stc_contract_spgemm", "stc_contract_spmm", "stc_contract_spmv",
                     "stc_bellman_ford", "stc_create", "stc_destroy", "stc_status_str"]:
        assert required in names


def test_every_declared_symbol_is_exported(libstc):
    names = declared_functions()
    assert names
    for n in names:
        assert hasattr(libstc, n), n


def test_status_strings_and_version(libstc):
    libstc.stc_status_str.restype = ctypes.c_char_p
    libstc.stc_status_str.argtypes = [ctypes.c_int]
    assert libstc.stc_status_str(0) == b"ok"
    assert b"negative cycle" in libstc.stc_status_str(7)
    assert libstc.stc_status_str(99) == b"unknown status"
    assert libstc.stc_version() >= 100


def test_null_arguments_are_rejected_before_any_device_work(libstc):
    f = libstc.stc_contract_spgemm
    f.restype = ctypes.c_int
    assert f(None, 0, None, None, None, None, None) == 1  # STC_ERR_INVALID_ARG
    libstc.stc_bellman_ford.restype = ctypes.c_int
    assert libstc.stc_bellman_ford(None, 2, None, 0, None, None, 1, None) == 1


def test_learned_and_tensor_core_entry_points_check_arguments_first(libstc):
    """Null handles, weights, buffers and negative sizes are rejected with
    STC_ERR_INVALID_ARG before any device work, for the perceptron entry points
    (CUDA-core and tensor-core forward) and the masked product."""
    p, i64 = ctypes.c_void_p, ctypes.c_int64
    for name in ("stc_mlp_forward", "stc_mlp_forward_tc"):
        f = getattr(libstc, name)
        f.restype = ctypes.c_int
        f.argtypes = [p, p, p, i64, p, p]
        assert f(None, None, None, 0, None, None) == 1
        dummy = ctypes.c_float(0.0)
        ptr = ctypes.addressof(dummy)
        assert f(None, ptr, ptr, 1, ptr, None) == 1      # no handle
        assert f(ptr, None, ptr, 1, ptr, None) == 1      # no weights
        assert f(ptr, ptr, None, 1, ptr, None) == 1      # rows without features
        assert f(ptr, ptr, ptr, -1, ptr, None) == 1      # negative row count
    g = libstc.stc_contract_spgemm_masked
    g.restype = ctypes.c_int
    assert g(None, 0, None, None, None, None, None, None) == 1

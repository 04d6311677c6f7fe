"""Host-side checks of the C ABI (no GPU): the library builds, loads and
exports every symbol include/dealias.h declares; host argument checks and
planning queries that need no device."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def lib():
    from paper_1008_1366_gb300 import _native, build
    build.build()
    return _native.load()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(dc_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ["dc_conv_complex_1d", "dc_conv_hermitian_1d", "dc_conv_ternary_hermitian_1d",
                 "dc_conv_complex_1d_batched", "dc_conv_complex_1d_adjoint"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    from paper_1008_1366_gb300 import _native
    assert set(declared_symbols()) <= set(_native.SIGNATURES)


def test_status_strings(lib):
    for code in range(8):
        assert lib.dc_status_string(code)
    assert lib.dc_status_string(99) == b"unknown status"


def test_null_and_bad_dtype_rejected_without_gpu(lib):
    # argument checks run before any CUDA call
    assert lib.dc_conv_complex_1d(None, None, None, 16, 0, None, 0, None) == 1
    p = ctypes.c_void_p(4096)
    assert lib.dc_conv_complex_1d(p, p, ctypes.c_void_p(8192), 16, 7, p, 1 << 20, None) == 1
    assert lib.dc_conv_complex_1d(p, p, ctypes.c_void_p(8192), -3, 0, p, 1 << 20, None) == 1
    # misaligned complex128 pointer
    assert lib.dc_conv_complex_1d(ctypes.c_void_p(4104), p, ctypes.c_void_p(8192), 16, 1, p, 1 << 20, None) == 3
    # partial overlap of output and input
    assert lib.dc_conv_complex_1d(p, ctypes.c_void_p(1 << 20), ctypes.c_void_p(4096 + 64), 16, 0, p, 1 << 20, None) == 1

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


def _ws(lib, kind, dims, dtype=0):
    d = (ctypes.c_int64 * len(dims))(*dims)
    out = ctypes.c_size_t(0)
    return lib.dc_workspace_size(kind, len(dims), d, dtype, ctypes.byref(out))


def test_sizes_with_repeated_odd_factors_are_planned(lib):
    # m = 2^a 3^b 5^c: odd Hermitian lengths (Sec. 2.3) and repeated odd
    # factors are planned; other primes are refused with DC_ERR_SIZE
    for m in [9, 15, 25, 27, 45, 75, 81, 125, 135, 225, 243, 405, 18, 90, 720, 2880, 3600, 9216, 12800]:
        for dtype in (0, 1):
            assert _ws(lib, 1, [m], dtype) == 0, (m, dtype)
            assert _ws(lib, 0, [m], dtype) == 0, (m, dtype)
    for m in [7, 11, 13, 49, 77, 1001]:
        assert _ws(lib, 1, [m]) == 2, m
    for dims in [[9, 15], [15, 45], [45, 12], [3, 9, 5], [27, 75]]:
        assert _ws(lib, 1, dims) == 0, dims
        assert _ws(lib, 0, dims) == 0, dims

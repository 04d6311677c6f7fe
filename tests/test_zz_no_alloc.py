"""dc_conv_complex_1d_noalloc: the 1D complex convolution for callers that
cannot allocate device memory (it uses a fixed scratch array inside the
library instead of a caller workspace).  Its output must match the
allocating entry point, dc_conv_complex_1d, on two calls in a row (the
shared array keeps the previous call's contents), and sizes beyond its
fixed scratch must be refused.  This file is collected last."""

import ctypes

import numpy as np
import pytest
import torch

from conftest import FP64_TOL, fp32_tol, rel_l2
from paper_1008_1366_gb300 import synthetic

pytestmark = pytest.mark.gpu

# (dtype, m): the two largest sizes use the two-level path and its scratch slot
CASES = [(torch.complex128, 16384), (torch.complex128, 20480), (torch.complex64, 40960),
         (torch.complex64, 1024), (torch.complex128, 96)]


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("dtype,m", CASES)
def test_noalloc_matches_allocating_entry_point(dtype, m):
    import paper_1008_1366_gb300 as dc
    from paper_1008_1366_gb300 import _native
    lib = _native.lib()
    code = 1 if dtype == torch.complex128 else 0
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    f = torch.tensor(synthetic.uniform_complex(m, 31 + m), dtype=dtype, device="cuda")
    g = torch.tensor(synthetic.uniform_complex(m, 41 + m), dtype=dtype, device="cuda")
    ref = dc.conv_complex_1d(f, g).cpu().numpy()
    tol = FP64_TOL if dtype == torch.complex128 else fp32_tol(2 * m)
    for _ in range(2):
        h = torch.full_like(f, complex(7.0, -7.0))
        st = lib.dc_conv_complex_1d_noalloc(_vp(f), _vp(g), _vp(h), m, code, stream)
        assert st == 0, lib.dc_status_string(st)
        torch.cuda.synchronize()
        assert rel_l2(h.cpu().numpy(), ref) <= tol


def test_noalloc_refuses_sizes_beyond_its_scratch():
    from paper_1008_1366_gb300 import _native
    lib = _native.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for code, dtype, m in ((1, torch.complex128, 24576), (0, torch.complex64, 49152)):
        t = torch.zeros(m, dtype=dtype, device="cuda")
        out = torch.zeros_like(t)
        assert lib.dc_conv_complex_1d_noalloc(_vp(t), _vp(t), _vp(out), m, code, stream) == 2

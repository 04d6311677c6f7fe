"""GPU parity of general implicit padding (Sec. 2.4: p m data modes zero
padded to N = q m, q sub-transforms of size m of p-term sums) against the
FP64 oracle, both precisions, both error bars of conftest.check_parity:
the full 2m - 1 outputs of the linear convolution (p = 1, q = 2), other
p/q rules with q >= 2p (full linear convolution), q < 2p (outputs wrapping
modulo qm), and the argument checks."""

import ctypes

import numpy as np
import pytest
import torch

import oracle
from conftest import check_parity, norm_scale

pytestmark = pytest.mark.gpu

from paper_1008_1366_gb300 import synthetic  # noqa: E402

DT = [torch.complex128, torch.complex64]


@pytest.fixture(scope="module")
def dc():
    import paper_1008_1366_gb300 as dc
    return dc


def dev(x, dtype):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


def ref_pq(f, g, m, q, nout):
    if len(f) * nout <= (1 << 22):
        return oracle.direct_complex_pq(f, g, m, q, nout)
    return oracle.padded_complex_pq(f, g, m, q, nout)


@pytest.mark.parametrize("m", [1, 2, 3, 8, 45, 64, 96, 640, 1024, 4096, 6144])
@pytest.mark.parametrize("dtype", DT)
def test_full_linear_output(dc, m, dtype):
    f = synthetic.uniform_complex(m, 40 + m)
    g = synthetic.uniform_complex(m, 41 + m)
    h = dc.conv_complex_1d_full(dev(f, dtype), dev(g, dtype)).cpu().numpy()
    assert h.shape == (2 * m - 1,)
    check_parity(h, ref_pq(f, g, m, 2, 2 * m - 1), dtype, 2 * m, norm_scale(f, g))
    # its first m outputs are the dealiased convolution of Sec. 2.1
    h1 = dc.conv_complex_1d(dev(f, dtype), dev(g, dtype)).cpu().numpy()
    check_parity(h[:m], h1, dtype, 2 * m, norm_scale(f, g))


PQ = [(64, 1, 3, None), (80, 2, 5, None), (64, 3, 7, None), (96, 1, 4, None), (256, 2, 3, None),
      (125, 2, 3, None), (48, 3, 4, None), (32, 5, 16, None), (512, 1, 2, 100), (512, 2, 3, 1536),
      (1024, 3, 5, 4000), (9, 4, 9, None), (2048, 1, 3, None)]


@pytest.mark.parametrize("m,p,q,nout", PQ)
@pytest.mark.parametrize("dtype", DT)
def test_pq_rules(dc, m, p, q, nout, dtype):
    f = synthetic.uniform_complex(p * m, 42 + m)
    g = synthetic.uniform_complex(p * m, 43 + m)
    h = dc.conv_complex_1d_pq(dev(f, dtype), dev(g, dtype), m, p, q, nout).cpu().numpy()
    n = nout if nout is not None else (2 * p * m - 1 if q >= 2 * p else q * m)
    assert h.shape == (n,)
    check_parity(h, ref_pq(f, g, m, q, n), dtype, q * m, norm_scale(f, g))


def test_pq_argument_checks(dc):
    from paper_1008_1366_gb300 import _native
    L = _native.lib()
    t = torch.zeros(1024, dtype=torch.complex64, device="cuda")
    o = torch.zeros(4096, dtype=torch.complex64, device="cuda")
    w = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    vp = lambda x: ctypes.c_void_p(x.data_ptr())
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.dc_conv_complex_1d_pq(vp(t), vp(t), vp(o), 512, 3, 2, 100, 0, vp(w), w.numel(), s) == 1    # q < p
    assert L.dc_conv_complex_1d_pq(vp(t), vp(t), vp(o), 512, 1, 2, 1025, 0, vp(w), w.numel(), s) == 1   # nout > qm
    assert L.dc_conv_complex_1d_pq(vp(t), vp(t), vp(o), 512, 1, 17, 100, 0, vp(w), w.numel(), s) == 1   # q > 16
    assert L.dc_conv_complex_1d_pq(vp(t), vp(t), vp(o), 7 * 64, 1, 2, 100, 0, vp(w), w.numel(), s) == 2  # 7 | m
    assert L.dc_conv_complex_1d_pq(vp(t), vp(t), vp(o), 512, 1, 2, 1023, 0, vp(w), 64, s) == 6          # workspace
    sz = ctypes.c_size_t(0)
    assert L.dc_workspace_size_pq(512, 1, 2, 1023, 0, ctypes.byref(sz)) == 0 and sz.value >= 2 * 1023 * 8

"""GPU parity at sizes with repeated odd factors, m = 2^a 3^b 5^c: the odd
Hermitian lengths m = 2c + 1 the paper allows (Sec. 2.3: odd m needs only
minor changes), and odd or non-power-of-two axes in 2D and 3D (Sec. 3.2,
Sec. 3.4), in both precisions, against the FP64 oracle with both error bars
of conftest.check_parity.  Lengths whose factors include both 3 and 5 run
as direct DFTs up to 512 and as two factors with one odd prime each above."""

import numpy as np
import pytest
import torch

import oracle
from conftest import check_parity, hermitian_scale, norm_scale
from oracle.adjoint import symmetrize_upstream
from paper_1008_1366_gb300 import synthetic

pytestmark = pytest.mark.gpu

DT = [torch.complex128, torch.complex64]
ODD = [9, 15, 25, 27, 45, 75, 81, 125, 135, 225, 243, 405]
EVEN = [18, 36, 50, 90, 144, 360, 720, 2880, 3600, 9216, 12800]


@pytest.fixture(scope="module")
def dc():
    import paper_1008_1366_gb300 as dc
    return dc


def dev(x, dtype):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


@pytest.mark.parametrize("m", ODD + EVEN)
@pytest.mark.parametrize("dtype", DT)
def test_hermitian_1d(dc, m, dtype):
    f = synthetic.hermitian_spectrum((m,), 1.0, 900 + m)
    g = synthetic.hermitian_spectrum((m,), 1.0, 901 + m)
    h = dc.conv_hermitian_1d(dev(f, dtype), dev(g, dtype)).cpu().numpy()
    check_parity(h, oracle.conv_hermitian(f, g), dtype, 3 * m, hermitian_scale(f, g))


@pytest.mark.parametrize("m", ODD + EVEN)
@pytest.mark.parametrize("dtype", DT)
def test_complex_1d(dc, m, dtype):
    f = synthetic.uniform_complex(m, 902 + m)
    g = synthetic.uniform_complex(m, 903 + m)
    h = dc.conv_complex_1d(dev(f, dtype), dev(g, dtype)).cpu().numpy()
    check_parity(h, oracle.conv_complex(f, g), dtype, 2 * m, norm_scale(f, g))


@pytest.mark.parametrize("m", [9, 15, 25, 45, 75, 135, 18, 90, 720])
@pytest.mark.parametrize("dtype", DT)
def test_ternary_1d(dc, m, dtype):
    f, g, e = (synthetic.hermitian_spectrum((m,), 1.0, s + m) for s in (904, 905, 906))
    h = dc.conv_ternary_hermitian_1d(dev(f, dtype), dev(g, dtype), dev(e, dtype)).cpu().numpy()
    check_parity(h, oracle.conv_ternary_hermitian(f, g, e), dtype, 4 * m, hermitian_scale(f, g, e))


@pytest.mark.parametrize("m", [9, 45, 225, 360])
@pytest.mark.parametrize("dtype", DT)
def test_hermitian_1d_adjoint(dc, m, dtype):
    f = synthetic.hermitian_spectrum((m,), 1.0, 907)
    g = synthetic.hermitian_spectrum((m,), 1.0, 908)
    w = synthetic.uniform_complex(m, 909)
    rdf, rdg = oracle.adjoint_hermitian(w, f, g)
    df, dg = dc.conv_hermitian_1d_adjoint(dev(w, dtype), dev(f, dtype), dev(g, dtype))
    W = symmetrize_upstream(w)
    check_parity(df.cpu().numpy(), rdf, dtype, 3 * m, hermitian_scale(W, g))
    check_parity(dg.cpu().numpy(), rdg, dtype, 3 * m, hermitian_scale(W, f))


H2 = [(9, 15), (15, 45), (5, 27), (45, 9), (25, 16), (16, 25), (9, 144), (27, 75)]


@pytest.mark.parametrize("ms", H2)
@pytest.mark.parametrize("dtype", DT)
def test_hermitian_2d(dc, ms, dtype):
    shape = synthetic.hermitian_shape(ms)
    f = synthetic.hermitian_spectrum(shape, 1.5, 910)
    g = synthetic.hermitian_spectrum(shape, 1.5, 911)
    h = dc.conv_hermitian_nd(dev(f, dtype), dev(g, dtype)).cpu().numpy()
    check_parity(h, oracle.padded_hermitian(f, g), dtype, np.prod([3 * m for m in ms]), hermitian_scale(f, g))


@pytest.mark.parametrize("shape", [(9, 15), (45, 12), (25, 27), (15, 9, 5)])
@pytest.mark.parametrize("dtype", DT)
def test_complex_nd(dc, shape, dtype):
    f = synthetic.uniform_complex(shape, 912)
    g = synthetic.uniform_complex(shape, 913)
    h = dc.conv_complex_nd(dev(f, dtype), dev(g, dtype)).cpu().numpy()
    check_parity(h, oracle.padded_complex(f, g), dtype, np.prod([2 * m for m in shape]), norm_scale(f, g))


@pytest.mark.parametrize("ms,spc", [((3, 9, 5), None), ((5, 3, 15), 4), ((9, 5, 9), 7)])
@pytest.mark.parametrize("dtype", DT)
def test_hermitian_3d(dc, ms, spc, dtype):
    shape = synthetic.hermitian_shape(ms)
    f = synthetic.hermitian_spectrum(shape, 11 / 6, 914)
    g = synthetic.hermitian_spectrum(shape, 11 / 6, 915)
    h = dc.conv_hermitian_nd(dev(f, dtype), dev(g, dtype), slabs_per_chunk=spc).cpu().numpy()
    check_parity(h, oracle.padded_hermitian(f, g), dtype, np.prod([3 * m for m in ms]), hermitian_scale(f, g))


@pytest.mark.parametrize("ms", [(9, 15), (5, 3, 9)])
@pytest.mark.parametrize("dtype", DT)
def test_hermitian_nd_adjoint(dc, ms, dtype):
    shape = synthetic.hermitian_shape(ms)
    f = synthetic.hermitian_spectrum(shape, 11 / 6, 916)
    g = synthetic.hermitian_spectrum(shape, 11 / 6, 917)
    w = synthetic.uniform_complex(shape, 918)
    rdf, rdg = oracle.adjoint_hermitian(w, f, g)
    df, dg = dc.conv_hermitian_nd_adjoint(dev(w, dtype), dev(f, dtype), dev(g, dtype))
    W = symmetrize_upstream(w)
    N = np.prod([3 * m for m in ms])
    check_parity(df.cpu().numpy(), rdf, dtype, N, hermitian_scale(W, g))
    check_parity(dg.cpu().numpy(), rdg, dtype, N, hermitian_scale(W, f))

"""Autograd: the backward kernels against torch.autograd.gradcheck (FP64,
small shapes), the FP64 oracle gradient (every output, both error bars of
conftest.check_parity, at the 3D benchmark shape too), and central finite
differences at the 3D benchmark shape."""

import numpy as np
import pytest
import torch

import oracle
from conftest import check_parity, hermitian_scale, rel_l2
from paper_1008_1366_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ag():
    from paper_1008_1366_gb300 import autograd
    return autograd


def dev(x, dtype=torch.complex128, grad=False):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda", requires_grad=grad)


@pytest.mark.parametrize("shape", [(6,), (16,), (4, 5), (3, 4, 4)])
def test_gradcheck_complex(ag, shape):
    f = dev(synthetic.uniform_complex(shape, 1), grad=True)
    g = dev(synthetic.uniform_complex(shape, 2), grad=True)
    assert torch.autograd.gradcheck(ag.conv_complex, (f, g), eps=1e-6, atol=1e-8, rtol=1e-6)


@pytest.mark.parametrize("ms", [(6,), (8,), (3, 4), (2, 2, 3)])
def test_gradcheck_hermitian(ag, ms):
    shape = synthetic.hermitian_shape(ms)
    f = dev(synthetic.uniform_complex(shape, 3), grad=True)
    g = dev(synthetic.uniform_complex(shape, 4), grad=True)
    assert torch.autograd.gradcheck(ag.conv_hermitian, (f, g), eps=1e-6, atol=1e-8, rtol=1e-6)


@pytest.mark.parametrize("ms", [(64,), (16, 12), (6, 6, 8), (4, 64), (2, 3, 96)])
def test_backward_matches_oracle_gradient(ag, ms):
    shape = synthetic.hermitian_shape(ms)
    f0 = synthetic.hermitian_spectrum(shape, 11 / 6, 5)
    g0 = synthetic.hermitian_spectrum(shape, 11 / 6, 6)
    w0 = synthetic.uniform_complex(shape, 7)
    f, g = dev(f0, grad=True), dev(g0, grad=True)
    h = ag.conv_hermitian(f, g)
    L = (h * dev(w0).conj()).sum().real
    L.backward()
    rdf, rdg = oracle.adjoint_hermitian(w0, f0, g0)
    from oracle.adjoint import symmetrize_upstream
    W = symmetrize_upstream(w0)
    N = int(np.prod([3 * m for m in ms]))
    check_parity(f.grad.cpu().numpy(), rdf, torch.complex128, N, hermitian_scale(W, g0))
    check_parity(g.grad.cpu().numpy(), rdg, torch.complex128, N, hermitian_scale(W, f0))


def test_hermitian_3d_256_backward(ag):
    """Forward and backward at 511 x 511 x 256 (complex64 data, FP64 tables):
    both gradients over every output against the FP64 oracle gradient (the
    padded oracle on a 768^3 grid), and a directional central difference
    (step 1e-3) of the FP64 path against Re <grad, v> within 1e-3."""
    ms = (256, 256, 256)
    shape = synthetic.hermitian_shape(ms)
    f0 = synthetic.hermitian_spectrum(shape, 11 / 6, 1021)
    g0 = synthetic.hermitian_spectrum(shape, 11 / 6, 1022)
    w0 = synthetic.uniform_complex(shape, 1023) * 1e-2
    f = dev(f0, torch.complex64, grad=True)
    g = dev(g0, torch.complex64, grad=True)
    h = ag.conv_hermitian(f, g)
    L = (h * dev(w0, torch.complex64).conj()).sum().real
    L.backward()
    df = f.grad.cpu().numpy()
    dg = g.grad.cpu().numpy()
    del f, g, h, L
    from oracle.adjoint import symmetrize_upstream
    W = symmetrize_upstream(w0)
    N = 27 * 256 ** 3
    rdf, rdg = oracle.adjoint_hermitian(w0, f0, g0)
    check_parity(df, rdf, torch.complex64, N, hermitian_scale(W, g0), what="df")
    check_parity(dg, rdg, torch.complex64, N, hermitian_scale(W, f0), what="dg")
    del rdf, rdg, dg
    # central difference in FP64 along a random direction
    v0 = (np.random.default_rng(2).uniform(-1, 1, shape) + 1j * np.random.default_rng(3).uniform(-1, 1, shape)) * 1e-2
    from paper_1008_1366_gb300 import api
    with torch.no_grad():
        f64, g64, w64, v64 = dev(f0), dev(g0), dev(w0), dev(v0)
        step = 1e-3
        Lp = (api.conv_hermitian_nd(f64 + step * v64, g64) * w64.conj()).sum().real.item()
        Lm = (api.conv_hermitian_nd(f64 - step * v64, g64) * w64.conj()).sum().real.item()
        fd = (Lp - Lm) / (2 * step)
        df64, _ = api.conv_hermitian_nd_adjoint(w64, f64, g64)
        an = (df64.conj() * v64).sum().real.item()
        an32 = float(np.real(np.vdot(df.astype(np.complex128), v0)))
    assert abs(fd - an) <= 1e-3 * abs(fd)
    assert abs(fd - an32) <= 1e-3 * abs(fd)

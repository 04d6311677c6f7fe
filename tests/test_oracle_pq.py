"""Pins of the general-padding oracles (Sec. 2.4: p m data modes zero padded
to N = q m; the convolution is the cyclic one of the padded arrays) against
facts outside them: numpy's polynomial product (the full linear convolution,
which N >= 2 p m - 1 leaves unaliased), the wrap-around of the linear
convolution modulo N when N is smaller, brute force of the cyclic sum with
Gaussian integers, and the closed form for constant inputs."""

import numpy as np
import pytest

import oracle
from conftest import gaussian_ints


@pytest.mark.parametrize("m,p,q", [(1, 1, 2), (3, 1, 2), (4, 1, 3), (5, 2, 5), (4, 3, 7), (6, 1, 4), (8, 2, 7)])
def test_full_linear_convolution_when_unaliased(m, p, q):
    # q >= 2p: N = q m >= 2 p m - 1, so the 2 p m - 1 outputs are the
    # coefficients of the product polynomial f(z) g(z)
    f = gaussian_ints(p * m, 1)
    g = gaussian_ints(p * m, 2)
    want = np.convolve(f, g)
    nout = 2 * p * m - 1
    assert np.array_equal(oracle.direct_complex_pq(f, g, m, q, nout), want)
    assert np.max(np.abs(oracle.padded_complex_pq(f, g, m, q, nout) - want)) < 1e-10
    # and the outputs beyond them are zero (no wave beats land there)
    if q * m > nout:
        tail = oracle.direct_complex_pq(f, g, m, q, q * m)[nout:]
        assert np.all(tail == 0)


@pytest.mark.parametrize("m,p,q", [(4, 2, 3), (5, 3, 4), (3, 2, 3), (6, 5, 6), (4, 3, 3)])
def test_aliased_outputs_wrap_modulo_N(m, p, q):
    # q < 2p: the padded DFTs alias the linear convolution modulo N = q m
    f = gaussian_ints(p * m, 3)
    g = gaussian_ints(p * m, 4)
    lin = np.convolve(f, g)
    N = q * m
    want = np.zeros(N, dtype=np.complex128)
    for k, v in enumerate(lin):
        want[k % N] += v
    assert np.array_equal(oracle.direct_complex_pq(f, g, m, q, N), want)
    assert np.max(np.abs(oracle.padded_complex_pq(f, g, m, q, N) - want)) < 1e-10


def test_constant_inputs_closed_form():
    # f = g = 1 on p m modes, N >= 2 p m - 1: h_k = min(k, 2 p m - 2 - k) + 1
    m, p, q = 7, 2, 5
    n = p * m
    f = np.ones(n)
    h = oracle.direct_complex_pq(f, f, m, q, 2 * n - 1)
    k = np.arange(2 * n - 1)
    assert np.array_equal(h, np.minimum(k, 2 * n - 2 - k) + 1)


def test_reduces_to_the_first_m_outputs_of_sec_2_1():
    # p = 1, q = 2: the first m outputs are the dealiased convolution of Sec. 2.1
    m = 12
    f = gaussian_ints(m, 5)
    g = gaussian_ints(m, 6)
    assert np.array_equal(oracle.direct_complex_pq(f, g, m, 2, m), oracle.direct_complex(f, g))

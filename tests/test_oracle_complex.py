"""Pins of the complex-convolution oracle (Sec. 2.1, Sec. 3.1, Sec. 3.4)
against facts outside the oracle: exact brute force, the paper's closed-form
error test, constants, geometric sequences, the polynomial-product identity
and separability."""

import itertools

import numpy as np
import pytest

import oracle
from conftest import gaussian_ints, rel_l2


def brute_complex_1d(f, g):
    m = len(f)
    return [sum(f[p] * g[k - p] for p in range(k + 1)) for k in range(m)]


def brute_complex_nd(f, g):
    shape = f.shape
    h = np.zeros(shape, dtype=np.complex128)
    for k in itertools.product(*[range(m) for m in shape]):
        s = 0
        for p in itertools.product(*[range(kk + 1) for kk in k]):
            q = tuple(kk - pp for kk, pp in zip(k, p))
            s += complex(f[p]) * complex(g[q])
        h[k] = s
    return h


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6, 8, 12, 16, 20, 24, 32, 48, 64])
def test_complex_1d_brute_force_exact(m):
    f = gaussian_ints(m, 10 + m)
    g = gaussian_ints(m, 20 + m)
    exact = brute_complex_1d([complex(x) for x in f], [complex(x) for x in g])
    # integer data: the direct sum is exact
    assert np.array_equal(oracle.direct_complex(f, g), np.array(exact))
    assert np.max(np.abs(oracle.padded_complex(f, g) - exact)) < 1e-11


@pytest.mark.parametrize("shape", [(1, 1), (2, 3), (4, 4), (5, 3), (8, 6), (2, 3, 4), (4, 4, 4), (3, 5, 2)])
def test_complex_nd_brute_force_exact(shape):
    f = gaussian_ints(shape, 1)
    g = gaussian_ints(shape, 2)
    exact = brute_complex_nd(f, g)
    assert np.array_equal(oracle.direct_complex(f, g), exact)
    assert np.max(np.abs(oracle.padded_complex(f, g) - exact)) < 1e-10


@pytest.mark.parametrize("m", [64, 1000, 1024, 4096])
def test_paper_closed_form_complex(m):
    # Sec. 2.1 error test: f_k = F e^{ik}, g_k = G e^{ik}, H_k = F G (k+1) e^{ik}
    F = np.sqrt(3) + 1j * np.sqrt(7)
    G = np.sqrt(5) + 1j * np.sqrt(11)
    k = np.arange(m)
    f = F * np.exp(1j * k)
    g = G * np.exp(1j * k)
    H = F * G * (k + 1) * np.exp(1j * k)
    assert rel_l2(oracle.direct_complex(f, g), H) < 1e-14
    assert rel_l2(oracle.padded_complex(f, g), H) < 1e-13


@pytest.mark.parametrize("shape", [(16,), (7, 9), (4, 5, 6)])
def test_constant_inputs_give_triangular(shape):
    f = np.ones(shape, dtype=np.complex128)
    expect = np.ones(shape)
    for a, m in enumerate(shape):
        sh = [1] * len(shape)
        sh[a] = m
        expect = expect * (np.arange(m) + 1).reshape(sh)
    assert np.array_equal(oracle.direct_complex(f, f), expect)
    assert np.max(np.abs(oracle.padded_complex(f, f) - expect)) < 1e-10


@pytest.mark.parametrize("a,b", [(0.9 + 0.1j, -0.5 + 0.7j), (0.99j, 0.99j), (1.01, 0.3)])
def test_geometric_closed_form(a, b):
    m = 300
    k = np.arange(m)
    f = a ** k
    g = b ** k
    if a == b:
        H = (k + 1) * a ** k
    else:
        H = (a ** (k + 1) - b ** (k + 1)) / (a - b)
    assert rel_l2(oracle.direct_complex(f, g), H) < 1e-13
    assert rel_l2(oracle.padded_complex(f, g), H) < 1e-12


@pytest.mark.parametrize("m", [1024, 2 ** 16, 3 * 2 ** 13])
def test_polynomial_identity_large(m):
    # With f, g supported on [0, m/2) the product polynomial has degree <= m-2,
    # so sum_{k<m} h_k z^k = f(z) g(z) exactly (polynomial multiplication).
    r = np.random.default_rng(m)
    f = np.zeros(m, complex)
    g = np.zeros(m, complex)
    f[: m // 2] = r.uniform(-1, 1, m // 2) + 1j * r.uniform(-1, 1, m // 2)
    g[: m // 2] = r.uniform(-1, 1, m // 2) + 1j * r.uniform(-1, 1, m // 2)
    h = oracle.padded_complex(f, g)
    for z in np.exp(2j * np.pi * r.uniform(size=4)):
        lhs = np.polyval(h[::-1], z)
        rhs = np.polyval(f[::-1], z) * np.polyval(g[::-1], z)
        assert abs(lhs - rhs) <= 1e-11 * np.sqrt(m) * max(1.0, abs(rhs))


@pytest.mark.parametrize("mx,my", [(6, 5), (16, 16), (64, 32)])
def test_separability_2d(mx, my):
    a = gaussian_ints(mx, 3) / 3
    b = gaussian_ints(my, 4) / 3
    c = gaussian_ints(mx, 5) / 3
    d = gaussian_ints(my, 6) / 3
    f = np.outer(a, b)
    g = np.outer(c, d)
    expect = np.outer(oracle.direct_complex(a, c), oracle.direct_complex(b, d))
    h = oracle.conv_complex(f, g)
    assert rel_l2(h, expect) < 1e-14
    assert rel_l2(oracle.padded_complex(f, g), expect) < 1e-13


def test_separability_3d():
    ax = [gaussian_ints(n, s) / 3 for n, s in ((5, 1), (6, 2), (4, 3))]
    bx = [gaussian_ints(n, s) / 3 for n, s in ((5, 4), (6, 5), (4, 6))]
    f = np.einsum("i,j,k->ijk", *ax)
    g = np.einsum("i,j,k->ijk", *bx)
    parts = [oracle.direct_complex(a, b) for a, b in zip(ax, bx)]
    expect = np.einsum("i,j,k->ijk", *parts)
    assert rel_l2(oracle.direct_complex(f, g), expect) < 1e-14
    assert rel_l2(oracle.padded_complex(f, g), expect) < 1e-13


def test_complex_at_matches_full():
    f = gaussian_ints((7, 9, 5), 11)
    g = gaussian_ints((7, 9, 5), 12)
    full = oracle.direct_complex(f, g)
    pts = [(0, 0, 0), (6, 8, 4), (3, 2, 1), (6, 0, 4)]
    assert np.array_equal(oracle.complex_at(f, g, pts), np.array([full[p] for p in pts]))


def test_numpy_fft_parseval():
    # the library FFT the padded oracle rests on: Parseval and round trip
    x = gaussian_ints(3 * 2 ** 10, 7)
    X = np.fft.fft(x)
    assert abs(len(x) * np.sum(abs(x) ** 2) - np.sum(abs(X) ** 2)) < 1e-9 * np.sum(abs(X) ** 2)
    assert np.max(abs(np.fft.ifft(X) - x)) < 1e-12


def test_oracle_fft_step_is_the_dft():
    # the padded oracle's library FFT step (scipy's threaded FFT where present):
    # the DFT by its definition on a small 3D grid (both signs, inverse scaled
    # by 1/N), then Parseval and the round trip at a size with factors 2, 3
    from oracle.conv import _fftn
    x = gaussian_ints((4, 6, 3), 8)
    n = x.shape
    ks = [np.arange(v) for v in n]
    W = [np.exp(-2j * np.pi * np.outer(k, k) / len(k)) for k in ks]
    X = np.einsum("ai,bj,ck,ijk->abc", W[0], W[1], W[2], x)
    assert np.max(abs(_fftn(x.copy()) - X)) < 1e-11
    Xi = np.einsum("ai,bj,ck,ijk->abc", W[0].conj(), W[1].conj(), W[2].conj(), x) / x.size
    assert np.max(abs(_fftn(x.copy(), inverse=True) - Xi)) < 1e-12
    y = gaussian_ints((48, 36), 9)
    Y = _fftn(y.copy())
    assert abs(y.size * np.sum(abs(y) ** 2) - np.sum(abs(Y) ** 2)) < 1e-9 * np.sum(abs(Y) ** 2)
    assert np.max(abs(_fftn(Y, inverse=True) - y)) < 1e-11


def test_golden_paper_closed_forms():
    # tests/golden/paper_closed_forms.txt: the exact solutions of the paper's
    # accuracy tests (Sec. 2.1 and Sec. 2.3) at m = 8
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_closed_forms.txt")
    rows = [ln.split() for ln in open(path) if not ln.startswith("#")]
    m = 8
    k = np.arange(m)
    e = np.exp(1j * k)
    cases = {
        "complex": oracle.direct_complex((np.sqrt(3) + 1j * np.sqrt(7)) * e, (np.sqrt(5) + 1j * np.sqrt(11)) * e),
        "hermitian": oracle.direct_hermitian(np.sqrt(3) * e, np.sqrt(5) * e),
    }
    for kind, kk, re, im in rows:
        assert abs(cases[kind][int(kk)] - complex(float(re), float(im))) < 1e-13

"""Pins of the M-pair (dot-product) oracles (Sec. 3, 2D pseudospectral
application: inputs as arrays of vectors, the product f * g read as
sum_i f_i * g_i) against the paper's worked example, the advective term of
the 2D Euler equation written out in Fourier space, and brute force."""

import itertools

import numpy as np
import pytest

import oracle
from conftest import gaussian_ints
from paper_1008_1366_gb300 import synthetic
from test_oracle_hermitian import brute_hermitian_nd, value_nd


def wave_vectors(shape):
    """(kx, ky) of every stored entry of a 2D Hermitian array (x centered)."""
    mx = (shape[0] + 1) // 2
    kx = np.arange(shape[0])[:, None] - (mx - 1) + 0 * np.arange(shape[1])[None, :]
    ky = 0 * np.arange(shape[0])[:, None] + np.arange(shape[1])[None, :]
    return kx, ky


def advective_brute(w):
    """sum_p (p_x k_y - p_y k_x) / |k - p|^2 w_p w_{k-p} at every stored k,
    over the box |p_d|, |k_d - p_d| <= m_d - 1 (terms with k = p vanish:
    the stream function has no zero mode)."""
    mx, my = (w.shape[0] + 1) // 2, w.shape[1]
    out = np.zeros(w.shape, dtype=np.complex128)
    for ix, iy in np.ndindex(*w.shape):
        k = (ix - (mx - 1), iy)
        s = 0
        for p in itertools.product(range(-mx + 1, mx), range(-my + 1, my)):
            q = (k[0] - p[0], k[1] - p[1])
            if abs(q[0]) > mx - 1 or abs(q[1]) > my - 1 or q == (0, 0):
                continue
            s += (p[0] * k[1] - p[1] * k[0]) / (q[0] ** 2 + q[1] ** 2) * value_nd(w, p) * value_nd(w, q)
        out[ix, iy] = s
    return out


@pytest.mark.parametrize("ms", [(2, 2), (3, 3), (4, 3), (3, 5)])
def test_euler_advective_term(ms):
    # the paper's call conv2(i kx w, i ky w, i ky w / k^2, -i kx w / k^2):
    # f = (i kx w, i ky w) is grad w, g = (i ky w / k^2, -i kx w / k^2) is
    # u = zhat x grad(del^-2 w), so sum_i f_i * g_i = u . grad w, the
    # negative of the displayed sum for -u . grad w
    shape = synthetic.hermitian_shape(ms)
    w = synthetic.hermitian_spectrum(shape, 1.5, 31)
    w = oracle.project_hermitian(w)
    kx, ky = wave_vectors(shape)
    k2 = (kx ** 2 + ky ** 2).astype(float)
    inv = np.where(k2 > 0, 1.0 / np.where(k2 > 0, k2, 1.0), 0.0)
    fs = [1j * kx * w, 1j * ky * w]
    gs = [1j * ky * w * inv, -1j * kx * w * inv]
    h = oracle.dot_hermitian(fs, gs)
    ref = -advective_brute(w)
    assert np.max(np.abs(h - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    assert np.max(np.abs(ref)) > 1e-3   # not a vacuous comparison


@pytest.mark.parametrize("ms", [(3,), (2, 3)])
def test_dot_hermitian_brute_force(ms):
    shape = synthetic.hermitian_shape(ms)
    fs = [gaussian_ints(shape, s) for s in (1, 2, 3)]
    gs = [gaussian_ints(shape, s) for s in (4, 5, 6)]
    if len(ms) == 1:
        fs = [f.reshape(1, -1) for f in fs]
        gs = [g.reshape(1, -1) for g in gs]
        exact = sum(brute_hermitian_nd(f, g) for f, g in zip(fs, gs)).reshape(-1)
        fs, gs = [f.reshape(-1) for f in fs], [g.reshape(-1) for g in gs]
    else:
        exact = sum(brute_hermitian_nd(f, g) for f, g in zip(fs, gs))
    assert np.max(np.abs(oracle.dot_hermitian(fs, gs) - exact)) < 1e-10


@pytest.mark.parametrize("shape", [(5,), (3, 4)])
def test_dot_complex_brute_force(shape):
    fs = [gaussian_ints(shape, s) for s in (7, 8)]
    gs = [gaussian_ints(shape, s) for s in (9, 10)]
    exact = np.zeros(shape, dtype=np.complex128)
    for k in np.ndindex(*shape):
        for i in range(2):
            for p in np.ndindex(*[kk + 1 for kk in k]):
                q = tuple(k[a] - p[a] for a in range(len(shape)))
                exact[k] += fs[i][p] * gs[i][q]
    assert np.max(np.abs(oracle.dot_complex(fs, gs) - exact)) < 1e-10


def test_single_pair_is_the_convolution():
    f, g = synthetic.uniform_complex(40, 1), synthetic.uniform_complex(40, 2)
    assert np.array_equal(oracle.dot_complex([f], [g]), oracle.conv_complex(f, g))
    with pytest.raises(ValueError):
        oracle.dot_hermitian([], [])

"""Pins of the centered Hermitian and ternary oracles (Sec. 2.3, Sec. 3.2,
Sec. 3.4, Sec. 4) against facts outside the oracle: brute force written from
the problem statement, the paper's closed-form test, the triple-count closed
form, Laurent-polynomial identities, symmetry and separability."""

import itertools
from math import comb

import numpy as np
import pytest

import oracle
from oracle.conv import _direct_box, hermitian_extend, project_hermitian
from paper_1008_1366_gb300 import synthetic
from conftest import gaussian_ints, rel_l2


# --- brute force from the problem statement (independent of oracle code) ----

def value_1d(f, p):
    """Wave number p of a stored 1D Hermitian vector: U_{-p} = conj(U_p),
    U_0 taken real (projection)."""
    if p == 0:
        return complex(f[0].real)
    if p > 0:
        return complex(f[p])
    return complex(f[-p]).conjugate()


def brute_hermitian_1d(f, g):
    m = len(f)
    return np.array([sum(value_1d(f, p) * value_1d(g, k - p) for p in range(k - m + 1, m))
                     for k in range(m)])


def brute_ternary_1d(f, g, e):
    m = len(f)
    out = []
    for k in range(m):
        s = 0
        for p in range(-m + 1, m):
            for q in range(-m + 1, m):
                r = k - p - q
                if -m < r < m:
                    s += value_1d(f, p) * value_1d(g, q) * value_1d(e, r)
        out.append(s)
    return np.array(out)


def value_nd(u, k):
    """Wave vector k of a stored nD Hermitian array (centered leading axes of
    2m-1 entries, last axis 0..m-1), with the self-conjugate row projected."""
    ms = [(n + 1) // 2 for n in u.shape[:-1]]
    def at(kk):
        return complex(u[tuple(kk[a] + ms[a] - 1 for a in range(len(ms))) + (kk[-1],)])
    neg = tuple(-x for x in k)
    if k[-1] > 0:
        return at(k)
    if k[-1] < 0:
        return at(neg).conjugate()
    return 0.5 * (at(k) + at(neg).conjugate())


def brute_hermitian_nd(f, g):
    ms = [(n + 1) // 2 for n in f.shape[:-1]] + [f.shape[-1]]
    rng_c = [range(-m + 1, m) for m in ms]
    out = np.zeros(f.shape, dtype=np.complex128)
    for idx in np.ndindex(*f.shape):
        k = [idx[a] - (ms[a] - 1) for a in range(len(ms) - 1)] + [idx[-1]]
        s = 0
        for p in itertools.product(*rng_c):
            q = [k[a] - p[a] for a in range(len(ms))]
            if all(abs(q[a]) <= ms[a] - 1 for a in range(len(ms))):
                s += value_nd(f, p) * value_nd(g, q)
        out[idx] = s
    return out


def brute_ternary_nd(f, g, e):
    """h_k = sum_{p+q+r=k} f_p g_q e_r over the box |p_d|, |q_d|, |r_d| <= m_d-1,
    at the stored wave vectors k, written out from the problem statement."""
    ms = [(n + 1) // 2 for n in f.shape[:-1]] + [f.shape[-1]]
    box = list(itertools.product(*[range(-m + 1, m) for m in ms]))
    out = np.zeros(f.shape, dtype=np.complex128)
    for idx in np.ndindex(*f.shape):
        k = [idx[a] - (ms[a] - 1) for a in range(len(ms) - 1)] + [idx[-1]]
        s = 0
        for p in box:
            fp = value_nd(f, p)
            for q in box:
                r = [k[a] - p[a] - q[a] for a in range(len(ms))]
                if all(abs(r[a]) <= ms[a] - 1 for a in range(len(ms))):
                    s += fp * value_nd(g, q) * value_nd(e, r)
        out[idx] = s
    return out


# --- 1D ----------------------------------------------------------------------

@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6, 8, 12, 16, 20, 32, 64])
def test_hermitian_1d_brute_force_exact(m):
    f = gaussian_ints(m, 30 + m)
    g = gaussian_ints(m, 40 + m)
    exact = brute_hermitian_1d(f, g)
    assert np.array_equal(oracle.direct_hermitian(f, g), exact)
    assert np.max(np.abs(oracle.padded_hermitian(f, g) - exact)) < 1e-10


@pytest.mark.parametrize("m", [64, 1000, 1024, 4096])
def test_paper_closed_form_hermitian(m):
    # Sec. 2.3 error test: F = sqrt 3, G = sqrt 5 real; H_k = F G (2m-1-k) e^{ik}
    k = np.arange(m)
    f = np.sqrt(3) * np.exp(1j * k)
    g = np.sqrt(5) * np.exp(1j * k)
    H = np.sqrt(15) * (2 * m - 1 - k) * np.exp(1j * k)
    assert rel_l2(oracle.direct_hermitian(f, g), H) < 1e-14
    assert rel_l2(oracle.padded_hermitian(f, g), H) < 1e-13


def test_constant_hermitian():
    m = 50
    one = np.ones(m, complex)
    assert np.array_equal(oracle.direct_hermitian(one, one).real, 2 * m - 1 - np.arange(m))


def laurent(coeffs_full, z):
    """sum_{k=-M}^{M} c_k z^k for c stored at index k+M."""
    M = (len(coeffs_full) - 1) // 2
    return np.polyval(coeffs_full[::-1], z) * z ** (-M)


@pytest.mark.parametrize("m", [2 ** 12, 2 ** 16])
def test_laurent_identity_hermitian_large(m):
    # f, g supported on |p| < m/2: the full product has |k| <= m-2, so the
    # stored half plus its mirror is the whole Laurent product F(z) G(z).
    u = synthetic.hermitian_spectrum((m,), 1.0, 5)
    v = synthetic.hermitian_spectrum((m,), 1.0, 6)
    u[m // 2:] = 0
    v[m // 2:] = 0
    h = oracle.padded_hermitian(u, v)
    hfull = np.concatenate([np.conj(h[:0:-1]), h])
    U, V = hermitian_extend(u), hermitian_extend(v)
    for z in np.exp(2j * np.pi * np.random.default_rng(m).uniform(size=4)):
        lhs = laurent(hfull, z)
        rhs = laurent(U, z) * laurent(V, z)
        assert abs(lhs - rhs) <= 1e-11 * np.sqrt(m) * max(1.0, abs(rhs))


def test_projection_properties():
    r = np.random.default_rng(3)
    for shape in [(7,), (7, 4), (5, 7, 3)]:
        a = r.normal(size=shape) + 1j * r.normal(size=shape)
        b = r.normal(size=shape) + 1j * r.normal(size=shape)
        Pa, Pb = project_hermitian(a), project_hermitian(b)
        assert np.allclose(project_hermitian(Pa), Pa, atol=0, rtol=1e-15)     # idempotent
        lhs = np.real(np.vdot(Pa, b))
        rhs = np.real(np.vdot(a, Pb))
        assert abs(lhs - rhs) < 1e-12                                          # self-adjoint
        s = synthetic.hermitian_spectrum(shape, 1.0, 9)
        assert np.allclose(project_hermitian(s), s, atol=1e-15)               # symmetric data fixed


# --- nD ------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(1, 1), (3, 2), (5, 3), (7, 4), (3, 3, 2), (5, 3, 3)])
def test_hermitian_nd_brute_force_exact(shape):
    f = gaussian_ints(shape, 7)
    g = gaussian_ints(shape, 8)
    exact = brute_hermitian_nd(f, g)
    assert np.array_equal(oracle.direct_hermitian(f, g), exact)
    assert np.max(np.abs(oracle.padded_hermitian(f, g) - exact)) < 1e-10


@pytest.mark.parametrize("shape", [(9, 6), (7, 5, 4)])
def test_hermitian_output_symmetry(shape):
    # the convolution over the full box of two Hermitian arrays is Hermitian
    f = synthetic.hermitian_spectrum(shape, 1.5, 1)
    g = synthetic.hermitian_spectrum(shape, 1.5, 2)
    F, G = hermitian_extend(f), hermitian_extend(g)
    ms = [(n + 1) // 2 for n in shape[:-1]] + [shape[-1]]
    lo = [-(m - 1) for m in ms]
    H = _direct_box(F, lo, G, lo, lo, F.shape)
    assert np.max(np.abs(H - np.conj(H[(slice(None, None, -1),) * H.ndim]))) < 1e-14
    h = oracle.direct_hermitian(f, g)
    assert np.max(np.abs(H[..., ms[-1] - 1:] - h)) < 1e-14


def _sym_full(n, seed):
    """A centered vector of 2n-1 entries with a(-k) = conj a(k)."""
    half = gaussian_ints(n, seed) / 2
    half[0] = half[0].real
    return np.concatenate([np.conj(half[:0:-1]), half])


@pytest.mark.parametrize("mx,my", [(4, 6), (8, 8), (16, 12)])
def test_separability_hermitian_2d(mx, my):
    a, c = _sym_full(mx, 1), _sym_full(mx, 2)
    b, d = gaussian_ints(my, 3) / 2, gaussian_ints(my, 4) / 2
    b[0], d[0] = b[0].real, d[0].real
    f, g = np.outer(a, b), np.outer(c, d)
    A = oracle.direct_hermitian(a[mx - 1:], c[mx - 1:])
    Afull = np.concatenate([np.conj(A[:0:-1]), A])
    expect = np.outer(Afull, oracle.direct_hermitian(b, d))
    assert rel_l2(oracle.direct_hermitian(f, g), expect) < 1e-14
    assert rel_l2(oracle.padded_hermitian(f, g), expect) < 1e-13


def test_separability_hermitian_3d():
    mx, my, mz = 4, 5, 6
    a, a2 = _sym_full(mx, 1), _sym_full(mx, 2)
    b, b2 = _sym_full(my, 3), _sym_full(my, 4)
    c, c2 = gaussian_ints(mz, 5) / 2, gaussian_ints(mz, 6) / 2
    c[0], c2[0] = c[0].real, c2[0].real
    f = np.einsum("i,j,k->ijk", a, b, c)
    g = np.einsum("i,j,k->ijk", a2, b2, c2)

    def full(u, v, n):
        h = oracle.direct_hermitian(u[n - 1:], v[n - 1:])
        return np.concatenate([np.conj(h[:0:-1]), h])

    expect = np.einsum("i,j,k->ijk", full(a, a2, mx), full(b, b2, my),
                       oracle.direct_hermitian(c, c2))
    assert rel_l2(oracle.direct_hermitian(f, g), expect) < 1e-14
    assert rel_l2(oracle.padded_hermitian(f, g), expect) < 1e-13


def test_hermitian_at_matches_full():
    f = synthetic.hermitian_spectrum((9, 7, 5), 11 / 6, 3)
    g = synthetic.hermitian_spectrum((9, 7, 5), 11 / 6, 4)
    full = oracle.direct_hermitian(f, g)
    pts = [(0, 0, 0), (8, 6, 4), (4, 3, 0), (2, 5, 1)]
    assert np.max(np.abs(oracle.hermitian_at(f, g, pts) - np.array([full[p] for p in pts]))) < 1e-15


# --- ternary ---------------------------------------------------------------

def triple_count(k, m):
    """#{(p,q,r) in [-m+1, m-1]^3 : p+q+r = k} by inclusion-exclusion on
    x_i = p_i + m - 1 in [0, 2m-2] summing to k + 3(m-1)."""
    s = k + 3 * (m - 1)
    tot = 0
    for j in range(4):
        t = s - j * (2 * m - 1)
        if t >= 0:
            tot += (-1) ** j * comb(3, j) * comb(t + 2, 2)
    return tot


@pytest.mark.parametrize("m", [1, 2, 3, 7])
def test_triple_count_formula(m):
    for k in range(m):
        brute = sum(1 for p in range(-m + 1, m) for q in range(-m + 1, m) if abs(k - p - q) <= m - 1)
        assert triple_count(k, m) == brute


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 8, 12])
def test_ternary_brute_force_exact(m):
    f, g, e = gaussian_ints(m, 1), gaussian_ints(m, 2), gaussian_ints(m, 3)
    exact = brute_ternary_1d(f, g, e)
    assert np.max(np.abs(oracle.direct_ternary_hermitian(f, g, e) - exact)) < 1e-11
    assert np.max(np.abs(oracle.padded_ternary_hermitian(f, g, e) - exact)) < 1e-10


@pytest.mark.parametrize("ms", [(2, 2), (2, 3), (3, 2), (3, 3), (2, 2, 2)])
def test_ternary_nd_brute_force_exact(ms):
    # the multi-D ternary case (the outer axes centered, the last one the
    # Hermitian half axis), on Gaussian integers so that the sums are exact
    shape = synthetic.hermitian_shape(ms)
    f, g, e = (gaussian_ints(shape, s) for s in (4, 5, 6))
    exact = brute_ternary_nd(f, g, e)
    assert np.max(np.abs(oracle.direct_ternary_hermitian(f, g, e) - exact)) < 1e-10
    assert np.max(np.abs(oracle.padded_ternary_hermitian(f, g, e) - exact)) < 1e-9


@pytest.mark.parametrize("m", [16, 256, 2 ** 14])
def test_ternary_closed_form(m):
    k = np.arange(m)
    Fc, Gc, Ec = np.sqrt(3), np.sqrt(5), np.sqrt(7)
    f, g, e = (c * np.exp(1j * k) for c in (Fc, Gc, Ec))
    H = Fc * Gc * Ec * np.array([triple_count(int(x), m) for x in k]) * np.exp(1j * k)
    h = oracle.conv_ternary_hermitian(f, g, e)
    assert rel_l2(h, H) < 1e-13


@pytest.mark.parametrize("m", [3 * 2 ** 10, 2 ** 14])
def test_laurent_identity_ternary_large(m):
    u, v, w = (synthetic.hermitian_spectrum((m,), 1.0, s) for s in (1, 2, 3))
    for x in (u, v, w):
        x[m // 3:] = 0
    h = oracle.padded_ternary_hermitian(u, v, w)
    hfull = np.concatenate([np.conj(h[:0:-1]), h])
    U, V, W = (hermitian_extend(x) for x in (u, v, w))
    for z in np.exp(2j * np.pi * np.random.default_rng(m).uniform(size=4)):
        lhs = laurent(hfull, z)
        rhs = laurent(U, z) * laurent(V, z) * laurent(W, z)
        assert abs(lhs - rhs) <= 1e-11 * np.sqrt(m) * max(1.0, abs(rhs))

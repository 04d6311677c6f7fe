"""Readings of the paper that the kernels rely on, checked in plain numpy
against the padded transforms they replace (no product code involved).

R-17: the ternary kind's N = 4m padding (Sec. 4.1) taken as four m-point
residues.  For centered data U_k, k = -m+1..m-1 (U_{-m} = 0), the backward
transform of the 4m-padded array at j = 4l + r equals the m-point
backward DFT over k = 0..m-1 of zeta_{4m}^{rk} (U_k + zeta_4^{-r} U_{k-m})
(with U_0 alone at k = 0), and the forward transform of any 4m-periodic
sequence u at wavenumber k (|k| < m) equals the sum over r of
zeta_{4m}^{-rk} S_r(k mod m), S_r the m-point forward DFT of u_{4l+r}.
The centered kind's three residues (Sec. 2.2, Eqs. (2.4)-(2.6)) are the
same statement with 3 for 4; both are checked."""

import numpy as np
import pytest


def zeta(n, e):
    return np.exp(2j * np.pi * np.asarray(e, dtype=float) / n)


def padded_backward(U, m, q):
    """Backward transform (exponent +) of the q m-padded array of U_k,
    k = -m+1..m-1, stored at index k mod qm."""
    N = q * m
    a = np.zeros(N, complex)
    for k in range(-m + 1, m):
        a[k % N] = U[k + m - 1]
    return np.fft.ifft(a) * N


def residue_inputs(U, m, q, r):
    """The fold of the residue form: zeta_{qm}^{rk} (U_k + zeta_q^{-r} U_{k-m})
    for k = 1..m-1, U_0 at k = 0 (U_{-m} = 0)."""
    w = np.zeros(m, complex)
    w[0] = U[m - 1]
    for k in range(1, m):
        w[k] = zeta(q * m, r * k) * (U[k + m - 1] + zeta(q, -r) * U[k - 1])
    return w


@pytest.mark.parametrize("q", [3, 4])
@pytest.mark.parametrize("m", [1, 2, 3, 5, 8, 12, 16])
def test_residue_form_of_the_backward_transform(q, m):
    rng = np.random.default_rng(1000 + 10 * q + m)
    U = rng.standard_normal(2 * m - 1) + 1j * rng.standard_normal(2 * m - 1)
    full = padded_backward(U, m, q)
    for r in range(q):
        # m-point backward DFT (exponent +), unnormalized
        u = np.fft.ifft(residue_inputs(U, m, q, r)) * m
        assert np.allclose(u, full[r::q], rtol=0, atol=1e-12 * max(1.0, np.abs(full).max()))


@pytest.mark.parametrize("q", [3, 4])
@pytest.mark.parametrize("m", [1, 2, 3, 5, 8, 12, 16])
def test_residue_form_of_the_forward_transform(q, m):
    rng = np.random.default_rng(2000 + 10 * q + m)
    N = q * m
    u = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    full = np.fft.fft(u)   # forward (exponent -), unnormalized
    S = [np.fft.fft(u[r::q]) for r in range(q)]
    for k in range(-m + 1, m):
        got = sum(zeta(N, -r * k) * S[r][k % m] for r in range(q))
        assert abs(got - full[k % N]) <= 1e-12 * max(1.0, np.abs(full).max())


def test_fold_factor_of_the_lower_half():
    # the forward output at k = kk - m is the kk output times zeta_q^r
    # (zeta_{qm}^{-r(kk-m)} = zeta_{qm}^{-r kk} zeta_q^{r}); for q = 4 that
    # factor is i^r, which the kernel applies by swapping components
    for q in (3, 4):
        m = 7
        for r in range(q):
            for kk in range(1, m):
                lhs = zeta(q * m, -r * (kk - m))
                rhs = zeta(q * m, -r * kk) * zeta(q, r)
                assert abs(lhs - rhs) < 1e-14
    for r in range(4):
        assert abs(zeta(4, r) - 1j ** r) < 1e-15
        assert abs(zeta(4, -r) - (-1j) ** r) < 1e-15

"""Plant plausible mistakes in the oracle (on the CPU) and check that the
pins reject each one: a dropped conjugate, a missing projection, a transposed
operand, too little padding, a wrong gradient sign or term."""

import numpy as np
import pytest

import oracle
import oracle.adjoint as oadj
import oracle.conv as oconv
from conftest import gaussian_ints, rel_l2
from test_oracle_complex import brute_complex_nd
from test_oracle_hermitian import brute_hermitian_1d, brute_hermitian_nd


def _paper_hermitian_ok(m=64):
    k = np.arange(m)
    f = np.sqrt(3) * np.exp(1j * k)
    g = np.sqrt(5) * np.exp(1j * k)
    H = np.sqrt(15) * (2 * m - 1 - k) * np.exp(1j * k)
    return rel_l2(oracle.direct_hermitian(f, g), H) < 1e-14


def test_planted_missing_conjugate_in_extension(monkeypatch):
    assert _paper_hermitian_ok()
    orig = oconv.hermitian_extend

    def bad(u):
        full = orig(u)
        m = u.shape[-1]
        full[..., : m - 1] = np.conj(full[..., : m - 1])   # drop the conj
        return full

    monkeypatch.setattr(oconv, "hermitian_extend", bad)
    assert not _paper_hermitian_ok()


def test_planted_missing_projection(monkeypatch):
    f, g = gaussian_ints((5, 3), 7), gaussian_ints((5, 3), 8)
    exact = brute_hermitian_nd(f, g)
    assert np.array_equal(oracle.direct_hermitian(f, g), exact)
    monkeypatch.setattr(oconv, "project_hermitian", lambda u: np.asarray(u, complex))
    assert not np.allclose(oracle.direct_hermitian(f, g), exact)


def test_planted_transposed_operand():
    f, g = gaussian_ints((4, 5), 1), gaussian_ints((5, 4), 2)
    exact = brute_complex_nd(f, g.T.copy())
    bad = oracle.direct_complex(f, g.reshape(4, 5))      # wrong axis order
    assert not np.allclose(bad, exact)


@pytest.mark.parametrize("kind", ["complex", "hermitian"])
def test_planted_short_padding(monkeypatch, kind):
    m = 16
    f, g = gaussian_ints(m, 3), gaussian_ints(m, 4)
    orig = oconv._padded_box

    def short(arrays, los, N, out_lo, out_shape):
        return orig(arrays, los, tuple(n - 3 for n in N), out_lo, out_shape)

    monkeypatch.setattr(oconv, "_padded_box", short)
    if kind == "complex":
        exact = np.array([sum(complex(f[p]) * complex(g[k - p]) for p in range(k + 1)) for k in range(m)])
        assert not np.allclose(oracle.padded_complex(f, g), exact)
    else:
        assert not np.allclose(oracle.padded_hermitian(f, g), brute_hermitian_1d(f, g))


def test_planted_gradient_without_conjugate(monkeypatch):
    r = np.random.default_rng(0)
    f, g, w = (r.normal(size=6) + 1j * r.normal(size=6) for _ in range(3))
    ref = oracle.grad_by_linearity(oracle.direct_complex, [f, g], 0, w)
    assert rel_l2(oracle.adjoint_complex(w, f, g)[0], ref) < 1e-13
    orig = oadj._correlate
    monkeypatch.setattr(oadj, "_correlate", lambda w_, g_, p: orig(w_, np.conj(g_), p))
    assert rel_l2(oracle.adjoint_complex(w, f, g)[0], ref) > 1e-3


def test_planted_gradient_without_symmetrization(monkeypatch):
    r = np.random.default_rng(1)
    f, g, w = (r.normal(size=(5, 3)) + 1j * r.normal(size=(5, 3)) for _ in range(3))
    ref = oracle.grad_by_linearity(oracle.direct_hermitian, [f, g], 0, w)
    assert rel_l2(oracle.adjoint_hermitian(w, f, g)[0], ref) < 1e-13
    monkeypatch.setattr(oadj, "symmetrize_upstream", lambda u: np.asarray(u, complex))
    assert rel_l2(oracle.adjoint_hermitian(w, f, g)[0], ref) > 1e-3

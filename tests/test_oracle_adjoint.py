"""Pins of the gradient oracle: closed forms against the literal definition
(gradient by linearity), the dot-product identity, and central finite
differences."""

import numpy as np
import pytest

import oracle
from paper_1008_1366_gb300 import synthetic
from conftest import rel_l2


def rnd(shape, seed):
    r = np.random.default_rng(seed)
    return r.normal(size=shape) + 1j * r.normal(size=shape)


@pytest.mark.parametrize("shape", [(1,), (5,), (9,), (3, 4), (2, 3, 3)])
def test_complex_adjoint_matches_definition(shape):
    f, g, w = rnd(shape, 1), rnd(shape, 2), rnd(shape, 3)
    df, dg = oracle.adjoint_complex(w, f, g, padded=False)
    assert rel_l2(df, oracle.grad_by_linearity(oracle.direct_complex, [f, g], 0, w)) < 1e-13
    assert rel_l2(dg, oracle.grad_by_linearity(oracle.direct_complex, [f, g], 1, w)) < 1e-13
    dfp, dgp = oracle.adjoint_complex(w, f, g, padded=True)
    assert rel_l2(dfp, df) < 1e-13 and rel_l2(dgp, dg) < 1e-13


@pytest.mark.parametrize("shape", [(1,), (4,), (7,), (5, 3), (3, 3, 2)])
def test_hermitian_adjoint_matches_definition(shape):
    # raw (non-symmetric) inputs: the projection is part of the map
    f, g, w = rnd(shape, 4), rnd(shape, 5), rnd(shape, 6)
    df, dg = oracle.adjoint_hermitian(w, f, g)
    assert rel_l2(df, oracle.grad_by_linearity(oracle.direct_hermitian, [f, g], 0, w)) < 1e-13
    assert rel_l2(dg, oracle.grad_by_linearity(oracle.direct_hermitian, [f, g], 1, w)) < 1e-13


@pytest.mark.parametrize("m", [1, 3, 6])
def test_ternary_adjoint_matches_definition(m):
    f, g, e, w = rnd(m, 7), rnd(m, 8), rnd(m, 9), rnd(m, 10)
    grads = oracle.adjoint_ternary_hermitian(w, f, g, e)
    for slot in range(3):
        ref = oracle.grad_by_linearity(oracle.direct_ternary_hermitian, [f, g, e], slot, w)
        assert rel_l2(grads[slot], ref) < 1e-13


@pytest.mark.parametrize("kind,shape", [("complex", (64,)), ("complex", (12, 10)),
                                        ("hermitian", (64,)), ("hermitian", (15, 8)),
                                        ("hermitian", (7, 7, 5))])
def test_dot_product_identity(kind, shape):
    # L is real-linear in f, so L(f) = Re <grad_f, f> (and likewise for g)
    f, g, w = rnd(shape, 11), rnd(shape, 12), rnd(shape, 13)
    if kind == "complex":
        h = oracle.conv_complex(f, g)
        df, dg = oracle.adjoint_complex(w, f, g)
    else:
        h = oracle.conv_hermitian(f, g)
        df, dg = oracle.adjoint_hermitian(w, f, g)
    L = oracle.loss(h, w)
    assert abs(L - np.real(np.vdot(df, f))) < 1e-12 * max(1, abs(L))
    assert abs(L - np.real(np.vdot(dg, g))) < 1e-12 * max(1, abs(L))


@pytest.mark.parametrize("shape", [(256,), (31, 16)])
def test_central_finite_differences(shape):
    f = synthetic.hermitian_spectrum(shape, 11 / 6, 1)
    g = synthetic.hermitian_spectrum(shape, 11 / 6, 2)
    w = rnd(shape, 3)
    v = np.random.default_rng(4).uniform(-1, 1, size=shape) + 1j * np.random.default_rng(5).uniform(-1, 1, size=shape)
    df, _ = oracle.adjoint_hermitian(w, f, g)
    step = 1e-3
    Lp = oracle.loss(oracle.conv_hermitian(f + step * v, g), w)
    Lm = oracle.loss(oracle.conv_hermitian(f - step * v, g), w)
    fd = (Lp - Lm) / (2 * step)
    assert abs(fd - np.real(np.vdot(df, v))) <= 1e-9 * max(1.0, abs(fd))

"""FP64 gradients of the dealiased convolutions (test infrastructure only).

The paper has no adjoint; the quantity is defined here from first principles.
For a real loss ``L = Re sum_k conj(w_k) h_k`` over the stored outputs, the
gradient with respect to a complex input x follows PyTorch's convention,
``grad_p = dL/d(Re x_p) + i dL/d(Im x_p)``.

``grad_by_linearity`` is that definition evaluated literally: every
convolution here is real-linear in each single input, so the partial
derivatives are the loss at unit inputs.  The closed forms below are derived
from it and pinned against it (tests/test_oracle_adjoint.py):

* complex (Sec. 2.1, Sec. 3.1): ``df_p = sum_{k>=p} w_k conj(g_{k-p})``, a
  correlation with the conjugate partner, and likewise dg.
* centered Hermitian (Sec. 2.3, Sec. 3.2): with W equal to w except on the
  self-conjugate row/plane (last-axis wavenumber 0), where
  ``W(k',0) = w(k',0) + conj(w(-k',0))``, the gradient is the Hermitian
  convolution of W with the partner, halved on that row/plane.
* ternary (Sec. 4): the same with the two partners.
"""

import numpy as np

from .conv import (
    _c,
    _flip_all,
    _direct_box,
    _padded_box,
    conv_hermitian,
    conv_ternary_hermitian,
)


def loss(h, w):
    """L = Re sum conj(w) h over the stored outputs."""
    return float(np.real(np.vdot(_c(w).ravel(), _c(h).ravel())))


def grad_by_linearity(fn, args, which, w):
    """Gradient of L(x) = Re <w, fn(args with x in slot `which`)> from its
    definition: L is real-linear in x, so dL/dRe x_p = L(e_p) and
    dL/dIm x_p = L(i e_p).  O(n) calls of fn: tiny sizes only."""
    x = _c(args[which])
    grad = np.zeros(x.shape, dtype=np.complex128)
    for idx in np.ndindex(*x.shape):
        vals = []
        for unit in (1.0, 1.0j):
            e = np.zeros(x.shape, dtype=np.complex128)
            e[idx] = unit
            a = list(args)
            a[which] = e
            vals.append(loss(fn(*a), w))
        grad[idx] = vals[0] + 1j * vals[1]
    return grad


def _correlate(w, g, padded):
    """c_p = sum_{k} w_k conj(g_{k-p}) for 0 <= p < m on every axis."""
    w, g = _c(w), _c(g)
    m = w.shape
    zero = [0] * w.ndim
    Gr = np.conj(_flip_all(g))           # index i <-> offset s = i - (m-1)
    loG = [-(n - 1) for n in m]
    if padded:
        return _padded_box([w, Gr], [zero, loG], tuple(2 * n for n in m), zero, m)
    return _direct_box(w, zero, Gr, loG, zero, m)


def adjoint_complex(w, f, g, padded=None):
    """(df, dg) for h = conv_complex(f, g) and upstream gradient w."""
    if padded is None:
        padded = int(np.prod(np.shape(w))) ** 2 > (1 << 22)
    return _correlate(w, g, padded), _correlate(w, f, padded)


def symmetrize_upstream(w):
    """W of the module docstring: w with its self-conjugate row/plane replaced
    by w(k',0) + conj(w(-k',0))."""
    W = _c(w).copy()
    row = W[..., 0]
    if row.ndim == 0:
        W[..., 0] = 2.0 * row.real
    else:
        W[..., 0] = row + np.conj(_flip_all(row))
    return W


def _halve_self_conjugate(x):
    x = x.copy()
    x[..., 0] *= 0.5
    return x


def adjoint_hermitian(w, f, g):
    """(df, dg) for h = conv_hermitian(f, g) (projection included)."""
    W = symmetrize_upstream(w)
    return (_halve_self_conjugate(conv_hermitian(W, g)),
            _halve_self_conjugate(conv_hermitian(W, f)))


def adjoint_ternary_hermitian(w, f, g, e):
    """(df, dg, de) for h = conv_ternary_hermitian(f, g, e)."""
    W = symmetrize_upstream(w)
    return (_halve_self_conjugate(conv_ternary_hermitian(W, g, e)),
            _halve_self_conjugate(conv_ternary_hermitian(W, f, e)),
            _halve_self_conjugate(conv_ternary_hermitian(W, f, g)))

"""Plain FP64 definitions of the dealiased convolutions (test infrastructure only).

Problem statements followed (Bowman & Roberts 2011):

* complex binary convolution, Sec. 2.1: inputs f, g of unpadded length m per
  axis with the Fourier origin at index 0; output
  ``h_k = sum_{p=0..k} f_p g_{k-p}`` for ``0 <= k < m`` (the quantity the
  error test of Sec. 2.1 compares against).  In d dimensions the same sum runs
  over every axis (Sec. 3.1, Sec. 3.4: N = 2m padding per axis).
* centered Hermitian convolution under the 2/3 rule, Sec. 1 and Sec. 2.3:
  inputs store the non-negative wavenumbers 0..m-1 of the last axis; the
  negative ones follow from ``U_{-k} = conj(U_k)``; output
  ``h_k = sum_{p=k-m+1}^{m-1} f_p g_{k-p}`` for ``0 <= k < m``.  In 2D/3D
  (Sec. 3.2, Sec. 3.4) the leading axes are centered and stored in full,
  ``2m-1`` entries with the origin at index ``m-1``; the symmetry reads
  ``U_{-k} = conj(U_k)`` for the whole wave vector; the sum runs over every p
  with both p and k-p inside the box ``|p_d| <= m_d - 1``.
* centered Hermitian ternary convolution, Sec. 4:
  ``h_k = sum_{p+q+r=k} f_p g_q e_r`` over ``p, q, r in [-m+1, m-1]``,
  ``0 <= k < m``.

Storage layout (row-major, last axis contiguous, Sec. 3.1):
  complex      1D (m,)  2D (mx, my)           3D (mx, my, mz)
  Hermitian    1D (m,)  2D (2mx-1, my)        3D (2mx-1, 2my-1, mz)

Reading of Sec. 5 (a prepackaged routine should enforce the Hermitian
symmetry of the stored data): before convolving, Hermitian inputs are mapped
by the orthogonal projection ``project_hermitian`` onto the symmetric subspace
(``U_0 <- Re U_0`` in 1D; ``U(k',0) <- (U(k',0) + conj U(-k',0))/2`` on the
last-axis-zero row/plane in 2D/3D).
"""

import os

import numpy as np

try:   # a threaded library FFT where scipy is present; numpy's otherwise
    import scipy.fft as _sfft
    FFT_LIBRARY = "scipy.fft"
except ImportError:   # pragma: no cover
    _sfft = None
    FFT_LIBRARY = "numpy.fft"


def _fftn(a, inverse=False):
    """Library n-dimensional DFT (a step of the padded convolution): numpy's
    sign and scaling conventions (forward e^{-2 pi i jk/N}, inverse with 1/N)."""
    if _sfft is not None:
        fn = _sfft.ifftn if inverse else _sfft.fftn
        return fn(a, workers=os.cpu_count() or 1, overwrite_x=True)
    return np.fft.ifftn(a) if inverse else np.fft.fftn(a)


def _c(a):
    return np.asarray(a, dtype=np.complex128)


def _flip_all(a):
    return a[(slice(None, None, -1),) * a.ndim]


# ---------------------------------------------------------------------------
# Hermitian storage helpers
# ---------------------------------------------------------------------------

def hermitian_half_sizes(shape):
    """Unpadded sizes m_d of a Hermitian storage shape: centered axes hold
    2m-1 entries, the last axis holds m."""
    ms = []
    for n in shape[:-1]:
        if n % 2 != 1:
            raise ValueError("centered Hermitian axes hold 2m-1 entries")
        ms.append((n + 1) // 2)
    ms.append(shape[-1])
    return tuple(ms)


def project_hermitian(u):
    """Orthogonal projection onto data obeying U_{-k} = conj(U_k) on the
    self-conjugate subspace (last-axis wavenumber 0).  Reading of Sec. 5."""
    u = _c(u).copy()
    row = u[..., 0]
    if row.ndim == 0:
        u[..., 0] = row.real
    else:
        # flipping every centered axis maps wavenumber k' to -k'
        u[..., 0] = 0.5 * (row + np.conj(_flip_all(row)))
    return u


def hermitian_extend(u):
    """Full centered array of a Hermitian storage array: every axis spans
    wavenumbers -m_d+1..m_d-1 with the origin at index m_d-1; entries with a
    negative last-axis wavenumber are conj(U(-k)) (Sec. 2.3, Sec. 3.2)."""
    u = _c(u)
    m_last = u.shape[-1]
    full = np.zeros(u.shape[:-1] + (2 * m_last - 1,), dtype=np.complex128)
    full[..., m_last - 1:] = u
    if m_last > 1:
        neg = np.conj(u[..., 1:])            # last-axis wavenumbers 1..m-1
        neg = neg[(slice(None, None, -1),) * (u.ndim - 1) + (slice(None),)]
        full[..., : m_last - 1] = neg[..., ::-1]   # position m-1-k holds -k
    return full


# ---------------------------------------------------------------------------
# generic box convolutions
# ---------------------------------------------------------------------------

def _direct_box(F, loF, G, loG, out_lo, out_shape):
    """h(k) = sum_p F(p) G(k-p), F stored for p in [loF, loF+n-1] per axis
    (array index p - loF), likewise G; output k in [out_lo, out_lo+shape-1]."""
    d = F.ndim
    hiF = [loF[a] + F.shape[a] - 1 for a in range(d)]
    hiG = [loG[a] + G.shape[a] - 1 for a in range(d)]
    h = np.zeros(out_shape, dtype=np.complex128)
    for kidx in np.ndindex(*out_shape):
        k = [out_lo[a] + kidx[a] for a in range(d)]
        a_ = [max(loF[a], k[a] - hiG[a]) for a in range(d)]
        b_ = [min(hiF[a], k[a] - loG[a]) for a in range(d)]
        if any(a_[x] > b_[x] for x in range(d)):
            continue
        fs = F[tuple(slice(a_[x] - loF[x], b_[x] - loF[x] + 1) for x in range(d))]
        # G(k-p) for p = a..b runs from index k-a-loG down to k-b-loG
        gs = G[tuple(slice(k[x] - b_[x] - loG[x], k[x] - a_[x] - loG[x] + 1)
                     for x in range(d))]
        h[kidx] = np.sum(fs * _flip_all(gs))
    return h


def _direct_box_at(F, loF, G, loG, points):
    """The sum of ``_direct_box`` at the listed output wave vectors only."""
    d = F.ndim
    hiF = [loF[a] + F.shape[a] - 1 for a in range(d)]
    hiG = [loG[a] + G.shape[a] - 1 for a in range(d)]
    out = np.zeros(len(points), dtype=np.complex128)
    for n, k in enumerate(points):
        a_ = [max(loF[a], k[a] - hiG[a]) for a in range(d)]
        b_ = [min(hiF[a], k[a] - loG[a]) for a in range(d)]
        if any(a_[x] > b_[x] for x in range(d)):
            continue
        fs = F[tuple(slice(a_[x] - loF[x], b_[x] - loF[x] + 1) for x in range(d))]
        gs = G[tuple(slice(k[x] - b_[x] - loG[x], k[x] - a_[x] - loG[x] + 1)
                     for x in range(d))]
        out[n] = np.sum(fs * _flip_all(gs))
    return out


def _padded_box(arrays, los, N, out_lo, out_shape):
    """Conventional explicitly zero-padded FFT convolution (Sec. 1): place each
    array at positions p mod N inside a zero array of shape N, multiply the
    DFTs, invert, and read the outputs at k mod N.  Correct whenever N is large
    enough that no wave beat wraps onto a requested output."""
    d = len(N)
    prod = None
    for A, lo in zip(arrays, los):
        P = np.zeros(N, dtype=np.complex128)
        idx = tuple((np.arange(A.shape[a]) + lo[a]) % N[a] for a in range(d))
        P[np.ix_(*idx)] = A
        T = _fftn(P)
        del P
        if prod is None:
            prod = T
        else:
            prod *= T
        del T
    H = _fftn(prod, inverse=True)
    oidx = tuple((np.arange(out_shape[a]) + out_lo[a]) % N[a] for a in range(d))
    return H[np.ix_(*oidx)]


# ---------------------------------------------------------------------------
# complex binary convolution (Sec. 2.1, Sec. 3.1, Sec. 3.4)
# ---------------------------------------------------------------------------

def direct_complex(f, g):
    """h_k = sum_{0<=p<=k} f_p g_{k-p} on every axis, 0 <= k < m (defining sum)."""
    f, g = _c(f), _c(g)
    assert f.shape == g.shape
    zero = [0] * f.ndim
    return _direct_box(f, zero, g, zero, zero, f.shape)


def padded_complex(f, g):
    """Same result by explicit zero padding to N = 2m per axis (Sec. 2.1)."""
    f, g = _c(f), _c(g)
    assert f.shape == g.shape
    zero = [0] * f.ndim
    return _padded_box([f, g], [zero, zero], tuple(2 * m for m in f.shape),
                       zero, f.shape)


def complex_at(f, g, points):
    """Defining sum at the listed output indices (tuples, 0 <= k_d < m_d)."""
    f, g = _c(f), _c(g)
    zero = [0] * f.ndim
    return _direct_box_at(f, zero, g, zero, [tuple(p) for p in points])


# ---------------------------------------------------------------------------
# centered Hermitian binary convolution (Sec. 2.3, Sec. 3.2, Sec. 3.4)
# ---------------------------------------------------------------------------

def _hermitian_out(ms):
    out_lo = [-(m - 1) for m in ms[:-1]] + [0]
    out_shape = tuple([2 * m - 1 for m in ms[:-1]] + [ms[-1]])
    return out_lo, out_shape


def direct_hermitian(f, g):
    """h_k = sum_p f_p g_{k-p} over the box |p_d|, |k_d-p_d| <= m_d-1, for the
    stored wave vectors k (last axis k >= 0), on the projected inputs."""
    ms = hermitian_half_sizes(np.shape(f))
    F = hermitian_extend(project_hermitian(f))
    G = hermitian_extend(project_hermitian(g))
    lo = [-(m - 1) for m in ms]
    out_lo, out_shape = _hermitian_out(ms)
    return _direct_box(F, lo, G, lo, out_lo, out_shape)


def padded_hermitian(f, g):
    """Same result by explicit zero padding of the full symmetric extension to
    N = 3m per axis (the 2/3 rule, Sec. 1; N >= 3m-2 suffices)."""
    ms = hermitian_half_sizes(np.shape(f))
    F = hermitian_extend(project_hermitian(f))
    G = hermitian_extend(project_hermitian(g))
    lo = [-(m - 1) for m in ms]
    out_lo, out_shape = _hermitian_out(ms)
    return _padded_box([F, G], [lo, lo], tuple(3 * m for m in ms), out_lo, out_shape)


def hermitian_at(f, g, points):
    """Defining Hermitian sum at listed stored output indices (array indices
    into the storage layout, not wave vectors)."""
    ms = hermitian_half_sizes(np.shape(f))
    F = hermitian_extend(project_hermitian(f))
    G = hermitian_extend(project_hermitian(g))
    lo = [-(m - 1) for m in ms]
    out_lo, _ = _hermitian_out(ms)
    ks = [tuple(int(p[a]) + out_lo[a] for a in range(len(ms))) for p in points]
    return _direct_box_at(F, lo, G, lo, ks)


# ---------------------------------------------------------------------------
# centered Hermitian ternary convolution (Sec. 4)
# ---------------------------------------------------------------------------

def direct_ternary_hermitian(f, g, e):
    """h_k = sum_{p+q+r=k} f_p g_q e_r over [-m+1, m-1]^3 per axis, stored k.
    The triple sum is taken as sum_r e_r (sum_{p+q=k-r} f_p g_q): the same
    terms grouped by r."""
    ms = hermitian_half_sizes(np.shape(f))
    F = hermitian_extend(project_hermitian(f))
    G = hermitian_extend(project_hermitian(g))
    E = hermitian_extend(project_hermitian(e))
    lo = [-(m - 1) for m in ms]
    lo2 = [-2 * (m - 1) for m in ms]
    FG = _direct_box(F, lo, G, lo, lo2, tuple(4 * m - 3 for m in ms))
    out_lo, out_shape = _hermitian_out(ms)
    return _direct_box(FG, lo2, E, lo, out_lo, out_shape)


def padded_ternary_hermitian(f, g, e):
    """Same result by explicit zero padding to N = 4m per axis (Sec. 4.1:
    N >= 4m-3 prevents the triple beats from wrapping)."""
    ms = hermitian_half_sizes(np.shape(f))
    arrs = [hermitian_extend(project_hermitian(a)) for a in (f, g, e)]
    lo = [-(m - 1) for m in ms]
    out_lo, out_shape = _hermitian_out(ms)
    return _padded_box(arrs, [lo, lo, lo], tuple(4 * m for m in ms), out_lo, out_shape)


# ---------------------------------------------------------------------------
# size-based dispatch used by the tests and the baseline legs
# ---------------------------------------------------------------------------

_DIRECT_LIMIT = 1 << 22     # output points x summands handled by direct sums


def conv_complex(f, g):
    n = int(np.prod(np.shape(f)))
    return direct_complex(f, g) if n * n <= _DIRECT_LIMIT else padded_complex(f, g)


def conv_hermitian(f, g):
    n = int(np.prod(np.shape(f)))
    return direct_hermitian(f, g) if n * n <= _DIRECT_LIMIT else padded_hermitian(f, g)


def conv_ternary_hermitian(f, g, e):
    n = int(np.prod(np.shape(f)))
    if n * n <= _DIRECT_LIMIT // 4:
        return direct_ternary_hermitian(f, g, e)
    return padded_ternary_hermitian(f, g, e)


# ---------------------------------------------------------------------------
# general padding (Sec. 2.4): p m data modes zero padded to N = q m
# ---------------------------------------------------------------------------

def direct_complex_pq(f, g, m, q, nout):
    """h_k = sum_{j} F_j G_{(k - j) mod N}, k < nout, for F, G the inputs
    (p m values each, p = len(f) / m) zero padded to N = q m: the cyclic
    convolution that the zero-padded DFTs of size q m compute (the
    definition the implicit p/q padding of Sec. 2.4 reproduces)."""
    f, g = _c(f), _c(g)
    N = q * m
    F = np.zeros(N, dtype=np.complex128)
    G = np.zeros(N, dtype=np.complex128)
    F[: len(f)] = f
    G[: len(g)] = g
    h = np.zeros(nout, dtype=np.complex128)
    for k in range(nout):
        j = np.arange(len(f))
        h[k] = np.sum(F[j] * G[(k - j) % N])
    return h


def padded_complex_pq(f, g, m, q, nout):
    """Same result by the explicitly zero-padded FFT convolution of size N = q m."""
    f, g = _c(f), _c(g)
    return _padded_box([f, g], [[0], [0]], (q * m,), [0], (nout,))


# ---------------------------------------------------------------------------
# inputs as arrays of vectors (Sec. 3, 2D pseudospectral application): the
# product f * g read as the dot product sum_i f_i * g_i of M pairs
# ---------------------------------------------------------------------------

def dot_complex(fs, gs):
    """sum_i conv_complex(f_i, g_i) over the M pairs (f_i, g_i)."""
    if len(fs) != len(gs) or not fs:
        raise ValueError("need M >= 1 pairs")
    return sum(conv_complex(f, g) for f, g in zip(fs, gs))


def dot_hermitian(fs, gs):
    """sum_i conv_hermitian(f_i, g_i) over the M pairs (f_i, g_i)."""
    if len(fs) != len(gs) or not fs:
        raise ValueError("need M >= 1 pairs")
    return sum(conv_hermitian(f, g) for f, g in zip(fs, gs))


"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws numbers: it holds none of the convolution arithmetic
and is shared by the tests, the oracle checks and the benchmark.  All draws
use numpy's PCG64 in float64; callers cast to complex64 where needed.

Recipes:
* ``uniform_complex``: real and imaginary parts i.i.d. uniform[-1, 1].
* ``hermitian_spectrum``: a centered Hermitian storage array (1D (m,),
  2D (2mx-1, my), 3D (2mx-1, 2my-1, mz)) with amplitude ``max(|k|, 1)**-alpha``
  (|k| the Euclidean norm of the integer wave vector) times a uniform random
  phase; the self-conjugate row/plane (last-axis wavenumber 0) is made
  symmetric by construction (``U(-k', 0) = conj U(k', 0)``, ``U(0) `` real), so
  the data already obey the symmetry a pseudospectral field has.
* ``batched_sizes``: sizes drawn uniformly from the 31 members of
  {2^k, 3*2^k, 5*2^k} in [64, 65536] (a discrete log-uniform law, since the
  members are nearly evenly spaced in log m).
* ``instance_inputs``: uniform[-1, 1] entries of chosen instances of a batch,
  each instance from its own seeded stream (a rank's share alone).
"""

import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def uniform_complex(shape, seed):
    r = rng(seed)
    re = r.uniform(-1.0, 1.0, size=shape)
    im = r.uniform(-1.0, 1.0, size=shape)
    return re + 1j * im


def _wavenumbers(shape):
    """Integer wave vectors of a Hermitian storage shape (centered leading axes,
    non-negative last axis), as a list of broadcastable arrays."""
    ks = []
    d = len(shape)
    for a, n in enumerate(shape):
        if a < d - 1:
            m = (n + 1) // 2
            k = np.arange(n) - (m - 1)
        else:
            k = np.arange(n)
        sh = [1] * d
        sh[a] = n
        ks.append(k.reshape(sh))
    return ks


def hermitian_spectrum(shape, alpha, seed):
    shape = tuple(int(s) for s in shape)
    r = rng(seed)
    ks = _wavenumbers(shape)
    k2 = sum(k.astype(np.float64) ** 2 for k in ks)
    amp = np.maximum(np.sqrt(k2), 1.0) ** (-float(alpha))
    phase = r.uniform(0.0, 2.0 * np.pi, size=shape)
    u = amp * np.exp(1j * phase)
    row = u[..., 0]
    if row.ndim == 0:
        u[..., 0] = amp[..., 0] * np.cos(phase[..., 0])
    else:
        flat = row.reshape(-1)            # C order: wave vector k' at i, -k' at n-1-i
        n = flat.size
        half = n // 2
        flat[:half] = np.conj(flat[::-1][:half])
        flat[half] = flat[half].real
        u[..., 0] = flat.reshape(row.shape)
    return u


def hermitian_shape(ms):
    """Storage shape for unpadded sizes (m_1, ..., m_d)."""
    ms = list(ms)
    return tuple([2 * m - 1 for m in ms[:-1]] + [ms[-1]])


SIZES_31 = sorted(
    [2 ** k for k in range(6, 17)]
    + [3 * 2 ** k for k in range(5, 15)]
    + [5 * 2 ** k for k in range(4, 14)]
)
assert len(SIZES_31) == 31 and SIZES_31[0] == 64 and SIZES_31[-1] == 65536


def batched_sizes(n, seed, sizes=None):
    sizes = SIZES_31 if sizes is None else sizes
    r = rng(seed)
    return np.asarray(sizes, dtype=np.int64)[r.integers(0, len(sizes), size=int(n))]


def instance_inputs(ms, ids, seed):
    """Packed f, g of the instances `ids` of a batch of sizes ms, with their
    offsets (len(ids)+1 entries).  Instance i draws its entries (real and
    imaginary parts uniform[-1, 1], f then g) from its own stream seeded by
    (seed, i), so a share of the batch is generated alone with the values it
    has in the whole batch."""
    sub = [int(ms[i]) for i in ids]
    off = np.zeros(len(sub) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sub)
    f = np.empty(int(off[-1]), dtype=np.complex128)
    g = np.empty(int(off[-1]), dtype=np.complex128)
    for k, i in enumerate(ids):
        r = np.random.Generator(np.random.PCG64([int(seed), int(i)]))
        m = sub[k]
        a, b = off[k], off[k + 1]
        f[a:b] = r.uniform(-1.0, 1.0, m) + 1j * r.uniform(-1.0, 1.0, m)
        g[a:b] = r.uniform(-1.0, 1.0, m) + 1j * r.uniform(-1.0, 1.0, m)
    return f, g, off


def batched_inputs(ms, seed):
    """Packed f, g for a batch of 1D complex instances of sizes ms, with the
    offsets array (n+1 entries)."""
    ms = np.asarray(ms, dtype=np.int64)
    off = np.zeros(len(ms) + 1, dtype=np.int64)
    off[1:] = np.cumsum(ms)
    tot = int(off[-1])
    f = uniform_complex(tot, seed)
    g = uniform_complex(tot, seed + 1)
    return f, g, off

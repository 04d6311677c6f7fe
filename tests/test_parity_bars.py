"""The two error bars of the GPU parity tests (conftest.check_parity), pinned
on the CPU: they accept a genuine FFT-based convolution computed in single
precision, and the pointwise bar rejects an error confined to a few small
outputs that the global relative L2 lets through."""

import numpy as np
import pytest

import oracle
from conftest import check_parity, hermitian_scale, norm_scale, rel_l2
from paper_1008_1366_gb300 import synthetic

sfft = pytest.importorskip("scipy.fft")


def fp32_padded_complex(f, g):
    """Explicitly padded FFT convolution of complex64 data in single precision."""
    m = len(f)
    F = np.zeros(2 * m, np.complex64)
    G = np.zeros(2 * m, np.complex64)
    F[:m] = f.astype(np.complex64)
    G[:m] = g.astype(np.complex64)
    h = sfft.ifft(sfft.fft(F) * sfft.fft(G))
    assert h.dtype == np.complex64
    return h[:m]


def fp32_padded_hermitian(f, g):
    """The same for the centered Hermitian convolution (full extension, N = 3m)."""
    m = len(f)
    Fx = oracle.hermitian_extend(oracle.project_hermitian(f)).astype(np.complex64)
    Gx = oracle.hermitian_extend(oracle.project_hermitian(g)).astype(np.complex64)
    N = 3 * m
    F = np.zeros(N, np.complex64)
    G = np.zeros(N, np.complex64)
    idx = (np.arange(2 * m - 1) - (m - 1)) % N
    F[idx] = Fx
    G[idx] = Gx
    h = sfft.ifft(sfft.fft(F) * sfft.fft(G))
    assert h.dtype == np.complex64
    return h[:m]


@pytest.mark.parametrize("m", [64, 1024, 16384, 65536])
def test_bars_accept_single_precision_fft_convolution(m):
    f = synthetic.uniform_complex(m, 1)
    g = synthetic.uniform_complex(m, 2)
    check_parity(fp32_padded_complex(f, g), oracle.conv_complex(f, g), np.complex64, 2 * m, norm_scale(f, g))
    u = synthetic.hermitian_spectrum((m,), 1.0, 3)
    v = synthetic.hermitian_spectrum((m,), 1.0, 4)
    check_parity(fp32_padded_hermitian(u, v), oracle.conv_hermitian(u, v), np.complex64, 3 * m,
                 hermitian_scale(u, v))


def test_pointwise_bar_catches_small_tail_error():
    # FP64 Hermitian convolution of a decaying spectrum: corrupt the eight
    # smallest outputs (about 1e-5 of the largest) by 5e-13 of the largest.
    # The global relative L2 stays below 1e-12; the pointwise bar does not.
    m = 4096
    u = synthetic.hermitian_spectrum((m,), 1.0, 5)
    v = synthetic.hermitian_spectrum((m,), 1.0, 6)
    ref = oracle.conv_hermitian(u, v)
    bad = ref.copy()
    tail = np.argsort(np.abs(ref))[:8]
    bad[tail] += 5e-13 * np.abs(ref).max()
    assert rel_l2(bad, ref) <= 1e-12
    with pytest.raises(AssertionError, match="pointwise"):
        check_parity(bad, ref, np.complex128, 3 * m, hermitian_scale(u, v))
    check_parity(ref, ref, np.complex128, 3 * m, hermitian_scale(u, v))


def test_ternary_scale_uses_l1_of_one_factor():
    a, b, c = (synthetic.uniform_complex(16, s) for s in (7, 8, 9))
    n2 = [np.linalg.norm(x) for x in (a, b, c)]
    n1 = [np.abs(x).sum() for x in (a, b, c)]
    want = n2[0] * n2[1] * n1[2] + n2[0] * n2[2] * n1[1] + n2[1] * n2[2] * n1[0]
    assert abs(norm_scale(a, b, c) - want) <= 1e-12 * want

import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def rel_l2(a, b):
    """Normalized L2 error of Sec. 2.1: ||a - b|| / ||b||."""
    a = np.asarray(a, dtype=np.complex128).ravel()
    b = np.asarray(b, dtype=np.complex128).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def fp32_tol(N):
    """Tolerance for the FP32 path: 5e-7 * log2(N), N the implicit padded size."""
    return 5e-7 * float(np.log2(N))


FP64_TOL = 1e-12


def gaussian_ints(shape, seed, lo=-3, hi=3):
    r = np.random.default_rng(seed)
    return (r.integers(lo, hi + 1, size=shape) + 1j * r.integers(lo, hi + 1, size=shape)).astype(np.complex128)


# ---------------------------------------------------------------------------
# pointwise error bar
# ---------------------------------------------------------------------------
# The global relative L2 above cannot see an error confined to a few outputs
# whose magnitude is far below the largest ones (spectra decaying like
# |k|^-alpha).  Every GPU parity test therefore also bounds each output's
# error.  A bound proportional to the local magnitude (|f| * |g|)_k does not
# hold for any FFT-based method: the rounding of the last transform is spread
# evenly over all outputs.  What does hold, for h = IFFT(FFT f . FFT g) / N
# with Cooley-Tukey transforms of normwise relative error eta log2 N (eta a
# few units of u with correctly rounded twiddles; Higham, Accuracy and
# Stability of Numerical Algorithms, Thm. 24.2):
#   |dh_k| <= eta log2N (2 ||f||_2 ||g||_2 + ||h_full||_2) + 2u ||f||_2 ||g||_2
# (Cauchy-Schwarz for the transformed inputs' errors, the normwise bound for
# the inverse transform).  For three factors the pointwise product costs an
# l1 norm: ||f||_2 ||g||_2 ||e||_1 and its permutations.  The implicit method
# computes the same padded transform factored into residues, so the same bar
# applies with N its padded size.  Input rounding to complex64 adds at most
# 2u ||f||_2 ||g||_2.  Taken here with eta = 8u and ||h_full|| <= 2 ||h||:
#   max_k |got_k - ref_k| <= 8 u log2(N) (2 S + 2 ||ref||_2) + 4u S.
# In FP64 this bar is about a thousand times tighter per output than the
# 1e-12 global one; in FP32 it is comparable to 5e-7 log2 N.
UNIT_ROUNDOFF = {"fp32": 2.0 ** -24, "fp64": 2.0 ** -53}


def precision_of(dtype):
    s = str(dtype)
    if "complex64" in s or "float32" in s:
        return "fp32"
    if "complex128" in s or "float64" in s:
        return "fp64"
    raise ValueError(f"unknown precision {dtype}")


def norm_scale(*arrays):
    """S of the pointwise bar: ||a||_2 ||b||_2 for two factors; for three the
    sum over which factor's transform error meets the other two's l1 norm."""
    arrs = [np.asarray(a, dtype=np.complex128).ravel() for a in arrays]
    n2 = [float(np.linalg.norm(a)) for a in arrs]
    if len(arrs) == 2:
        return n2[0] * n2[1]
    if len(arrs) == 3:
        n1 = [float(np.sum(np.abs(a))) for a in arrs]
        return n2[0] * n2[1] * n1[2] + n2[0] * n2[2] * n1[1] + n2[1] * n2[2] * n1[0]
    raise ValueError("one to three factors")


def hermitian_scale(*arrays):
    """norm_scale over the full symmetric extensions of Hermitian storage
    arrays (after the projection the convolution applies)."""
    import oracle
    return norm_scale(*[oracle.hermitian_extend(oracle.project_hermitian(a)) for a in arrays])


def pointwise_bound(ref, N, prec, scale):
    u = UNIT_ROUNDOFF[prec]
    nref = float(np.linalg.norm(np.asarray(ref, dtype=np.complex128).ravel()))
    return 8.0 * u * float(np.log2(max(N, 2))) * (2.0 * scale + 2.0 * nref) + 4.0 * u * scale


def check_parity(got, ref, dtype, N, scale, tol=None, what=""):
    """Both bars: relative L2 <= tol (default: 1e-12 FP64, 5e-7 log2 N FP32)
    and every output within the pointwise bar.  Returns (rel L2, max
    pointwise error / bar)."""
    prec = precision_of(dtype)
    t = tol if tol is not None else (FP64_TOL if prec == "fp64" else fp32_tol(N))
    got = np.asarray(got, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    e = rel_l2(got, ref)
    assert e <= t, f"{what} rel L2 {e:.3e} > {t:.3e}"
    bar = pointwise_bound(ref, N, prec, scale)
    pw = float(np.max(np.abs(got - ref))) if got.size else 0.0
    assert pw <= bar, f"{what} pointwise {pw:.3e} > {bar:.3e}"
    return e, pw / bar if bar > 0 else 0.0

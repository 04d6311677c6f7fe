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

"""GPU parity of the 2D/3D convolutions and their gradients against the FP64
oracle, through the C ABI.  Small shapes are compared element by element;
the full benchmark shapes against the padded oracle (2D) or direct sums at
sampled output points (3D)."""

import numpy as np
import pytest
import torch

import oracle
from conftest import FP64_TOL, fp32_tol, rel_l2
from paper_1008_1366_gb300 import synthetic

pytestmark = pytest.mark.gpu

DT = [torch.complex128, torch.complex64]


@pytest.fixture(scope="module")
def dc():
    import paper_1008_1366_gb300 as dc
    return dc


def dev(x, dtype):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


def tol(dtype, N):
    return FP64_TOL if dtype == torch.complex128 else fp32_tol(N)


C2 = [(1, 1), (2, 3), (4, 5), (8, 8), (16, 12), (3, 40), (32, 64), (64, 48)]
C3 = [(1, 1, 1), (2, 3, 4), (4, 4, 4), (8, 6, 5), (16, 16, 16), (5, 12, 8)]


@pytest.mark.parametrize("shape", C2 + C3)
@pytest.mark.parametrize("dtype", DT)
def test_complex_nd(dc, shape, dtype):
    f = synthetic.uniform_complex(shape, 1)
    g = synthetic.uniform_complex(shape, 2)
    h = dc.conv_complex_nd(dev(f, dtype), dev(g, dtype)).cpu().numpy()
    assert rel_l2(h, oracle.conv_complex(f, g)) <= tol(dtype, np.prod([2 * m for m in shape]))


H2 = [(1, 1), (2, 2), (3, 4), (8, 8), (16, 12), (5, 20), (32, 32), (64, 64)]
H3 = [(1, 1, 1), (2, 2, 2), (3, 4, 5), (4, 4, 4), (8, 8, 8), (6, 10, 12)]


@pytest.mark.parametrize("ms", H2 + H3)
@pytest.mark.parametrize("dtype", DT)
def test_hermitian_nd(dc, ms, dtype):
    shape = synthetic.hermitian_shape(ms)
    f = synthetic.hermitian_spectrum(shape, 1.5, 3)
    g = synthetic.hermitian_spectrum(shape, 1.5, 4)
    h = dc.conv_hermitian_nd(dev(f, dtype), dev(g, dtype)).cpu().numpy()
    assert rel_l2(h, oracle.conv_hermitian(f, g)) <= tol(dtype, np.prod([3 * m for m in ms]))


# outer axes of every length the compile-time outer-axis kernels cover
# (2^a, 64..4096; centered axes take 8 elements per thread up to 512)
OUTER_H = [(128, 4), (256, 3), (512, 2), (2048, 2), (4096, 2), (128, 3, 4), (3, 128, 4), (64, 64, 2)]
OUTER_C = [(128, 3), (256, 5), (512, 2), (1024, 2), (4096, 2), (128, 64, 2)]


@pytest.mark.parametrize("ms", OUTER_H)
@pytest.mark.parametrize("dtype", DT)
def test_hermitian_nd_outer_lengths(dc, ms, dtype):
    shape = synthetic.hermitian_shape(ms)
    f = synthetic.hermitian_spectrum(shape, 1.5, 15)
    g = synthetic.hermitian_spectrum(shape, 1.5, 16)
    h = dc.conv_hermitian_nd(dev(f, dtype), dev(g, dtype)).cpu().numpy()
    assert rel_l2(h, oracle.padded_hermitian(f, g)) <= tol(dtype, np.prod([3 * m for m in ms]))


@pytest.mark.parametrize("shape", OUTER_C)
@pytest.mark.parametrize("dtype", DT)
def test_complex_nd_outer_lengths(dc, shape, dtype):
    f = synthetic.uniform_complex(shape, 17)
    g = synthetic.uniform_complex(shape, 18)
    h = dc.conv_complex_nd(dev(f, dtype), dev(g, dtype)).cpu().numpy()
    assert rel_l2(h, oracle.padded_complex(f, g)) <= tol(dtype, np.prod([2 * m for m in shape]))


# wide rows: the row convolutions run on the fixed-shape engine (every
# size family, both precisions)
HW = [(2, 64), (2, 80), (3, 96), (2, 640), (2, 1536), (2, 4096), (2, 6144), (4, 5120), (2, 3, 256), (2, 8192),
      (3, 12288), (2, 20480), (2, 2, 16384)]


@pytest.mark.parametrize("ms", HW)
@pytest.mark.parametrize("dtype", DT)
def test_hermitian_nd_wide_rows(dc, ms, dtype):
    shape = synthetic.hermitian_shape(ms)
    f = synthetic.hermitian_spectrum(shape, 1.5, 13)
    g = synthetic.hermitian_spectrum(shape, 1.5, 14)
    h = dc.conv_hermitian_nd(dev(f, dtype), dev(g, dtype)).cpu().numpy()
    assert rel_l2(h, oracle.padded_hermitian(f, g)) <= tol(dtype, np.prod([3 * m for m in ms]))


@pytest.mark.parametrize("ms", [(4, 6), (3, 4, 5)])
def test_hermitian_nd_projects_raw_inputs(dc, ms):
    # inputs violating the symmetry on the self-conjugate row/plane are projected
    shape = synthetic.hermitian_shape(ms)
    f = synthetic.uniform_complex(shape, 5)
    g = synthetic.uniform_complex(shape, 6)
    h = dc.conv_hermitian_nd(dev(f, torch.complex128), dev(g, torch.complex128)).cpu().numpy()
    assert rel_l2(h, oracle.conv_hermitian(f, g)) <= FP64_TOL


@pytest.mark.parametrize("shape", [(3, 5), (16, 8), (4, 6, 5), (8, 8, 8)])
@pytest.mark.parametrize("dtype", DT)
def test_complex_nd_adjoint(dc, shape, dtype):
    w, f, g = (synthetic.uniform_complex(shape, s) for s in (7, 8, 9))
    rdf, rdg = oracle.adjoint_complex(w, f, g)
    df, dg = dc.conv_complex_nd_adjoint(dev(w, dtype), dev(f, dtype), dev(g, dtype))
    N = np.prod([2 * m for m in shape])
    assert rel_l2(df.cpu().numpy(), rdf) <= tol(dtype, N)
    assert rel_l2(dg.cpu().numpy(), rdg) <= tol(dtype, N)


# last axis 64 and up (one-level sizes of the set): the gradient rows run on
# the fixed-shape engine's pair residue
@pytest.mark.parametrize("ms", [(3, 4), (8, 8), (2, 3, 4), (4, 4, 6), (3, 64), (2, 96), (2, 3, 80), (2, 640),
                                (2, 4096), (2, 2, 256)])
@pytest.mark.parametrize("dtype", DT)
def test_hermitian_nd_adjoint(dc, ms, dtype):
    shape = synthetic.hermitian_shape(ms)
    f = synthetic.hermitian_spectrum(shape, 11 / 6, 10)
    g = synthetic.hermitian_spectrum(shape, 11 / 6, 11)
    w = synthetic.uniform_complex(shape, 12)
    rdf, rdg = oracle.adjoint_hermitian(w, f, g)
    df, dg = dc.conv_hermitian_nd_adjoint(dev(w, dtype), dev(f, dtype), dev(g, dtype))
    N = np.prod([3 * m for m in ms])
    assert rel_l2(df.cpu().numpy(), rdf) <= tol(dtype, N)
    assert rel_l2(dg.cpu().numpy(), rdg) <= tol(dtype, N)


# --- benchmark shapes -----------------------------------------------------------

def test_hermitian_2d_1024(dc):
    ms = (1024, 1024)
    shape = synthetic.hermitian_shape(ms)
    f = synthetic.hermitian_spectrum(shape, 1.5, 1011)
    g = synthetic.hermitian_spectrum(shape, 1.5, 1012)
    h = dc.conv_hermitian_nd(dev(f, torch.complex64), dev(g, torch.complex64)).cpu().numpy()
    assert rel_l2(h, oracle.padded_hermitian(f, g)) <= fp32_tol(9 * 1024 * 1024)


def test_complex_2d_2048(dc):
    f = synthetic.uniform_complex((2048, 2048), 1013)
    g = synthetic.uniform_complex((2048, 2048), 1014)
    h = dc.conv_complex_nd(dev(f, torch.complex64), dev(g, torch.complex64)).cpu().numpy()
    assert rel_l2(h, oracle.padded_complex(f, g)) <= fp32_tol(4 * 2048 * 2048)


def sampled_check(h, f, g, tol_, seed=0, nrand=8):
    """Full-size check from direct sums at sampled outputs: at the low
    wavenumbers (largest outputs) the per-point relative error; at uniformly
    random points an unbiased estimate of the global relative L2 error,
    sqrt(n * mean |err|^2) / ||h||."""
    shape = h.shape
    c = [(n - 1) // 2 for n in shape[:-1]]
    low = [tuple(c) + (0,), tuple(c) + (1,), (c[0] - 1, c[1] + 2, 3) if len(c) > 1 else (c[0] - 1, 3)]
    r = np.random.default_rng(seed)
    rnd = [tuple(int(r.integers(0, n)) for n in shape) for _ in range(nrand)]
    ref = oracle.hermitian_at(f, g, low + rnd)
    got = np.array([h[p] for p in low + rnd])
    err = np.abs(got - ref)
    per_point = err[: len(low)] / np.abs(ref[: len(low)])
    est = np.sqrt(h.size * np.mean(err[len(low):] ** 2)) / np.linalg.norm(h)
    return per_point, est


def test_hermitian_3d_256_sampled(dc):
    ms = (256, 256, 256)
    shape = synthetic.hermitian_shape(ms)
    f = synthetic.hermitian_spectrum(shape, 11 / 6, 1015)
    g = synthetic.hermitian_spectrum(shape, 11 / 6, 1016)
    h = dc.conv_hermitian_nd(dev(f, torch.complex64), dev(g, torch.complex64)).cpu().numpy()
    per_point, est = sampled_check(h, f, g, None)
    t = fp32_tol(27 * 256 ** 3)
    assert np.all(per_point <= t), per_point
    assert est <= t, est

"""GPU parity of the 2D/3D convolutions and their gradients against the FP64
oracle, through the C ABI.  Every output is compared (relative L2 and the
pointwise bar of conftest.check_parity): small shapes against the direct
sums, the full benchmark shapes (2D and 3D) against the explicitly padded
FP64 oracle, and 3D calls forced into several chunks of x-slabs with a
partial last chunk."""

import numpy as np
import pytest
import torch

import oracle
from conftest import FP64_TOL, check_parity, fp32_tol, hermitian_scale, norm_scale, rel_l2
from oracle.adjoint import symmetrize_upstream
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
    check_parity(h, oracle.conv_complex(f, g), dtype, np.prod([2 * m for m in shape]), norm_scale(f, g))


H2 = [(1, 1), (2, 2), (3, 4), (8, 8), (16, 12), (5, 20), (32, 32), (64, 64)]
H3 = [(1, 1, 1), (2, 2, 2), (3, 4, 5), (4, 4, 4), (8, 8, 8), (6, 10, 12)]


@pytest.mark.parametrize("ms", H2 + H3)
@pytest.mark.parametrize("dtype", DT)
def test_hermitian_nd(dc, ms, dtype):
    shape = synthetic.hermitian_shape(ms)
    f = synthetic.hermitian_spectrum(shape, 1.5, 3)
    g = synthetic.hermitian_spectrum(shape, 1.5, 4)
    h = dc.conv_hermitian_nd(dev(f, dtype), dev(g, dtype)).cpu().numpy()
    check_parity(h, oracle.conv_hermitian(f, g), dtype, np.prod([3 * m for m in ms]), hermitian_scale(f, g))


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
    check_parity(h, oracle.padded_hermitian(f, g), dtype, np.prod([3 * m for m in ms]), hermitian_scale(f, g))


@pytest.mark.parametrize("shape", OUTER_C)
@pytest.mark.parametrize("dtype", DT)
def test_complex_nd_outer_lengths(dc, shape, dtype):
    f = synthetic.uniform_complex(shape, 17)
    g = synthetic.uniform_complex(shape, 18)
    h = dc.conv_complex_nd(dev(f, dtype), dev(g, dtype)).cpu().numpy()
    check_parity(h, oracle.padded_complex(f, g), dtype, np.prod([2 * m for m in shape]), norm_scale(f, g))


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
    check_parity(h, oracle.padded_hermitian(f, g), dtype, np.prod([3 * m for m in ms]), hermitian_scale(f, g))


@pytest.mark.parametrize("ms", [(4, 6), (3, 4, 5)])
def test_hermitian_nd_projects_raw_inputs(dc, ms):
    # inputs violating the symmetry on the self-conjugate row/plane are projected
    shape = synthetic.hermitian_shape(ms)
    f = synthetic.uniform_complex(shape, 5)
    g = synthetic.uniform_complex(shape, 6)
    h = dc.conv_hermitian_nd(dev(f, torch.complex128), dev(g, torch.complex128)).cpu().numpy()
    check_parity(h, oracle.conv_hermitian(f, g), torch.complex128, np.prod([3 * m for m in ms]),
                 hermitian_scale(f, g))


@pytest.mark.parametrize("shape", [(3, 5), (16, 8), (4, 6, 5), (8, 8, 8)])
@pytest.mark.parametrize("dtype", DT)
def test_complex_nd_adjoint(dc, shape, dtype):
    w, f, g = (synthetic.uniform_complex(shape, s) for s in (7, 8, 9))
    rdf, rdg = oracle.adjoint_complex(w, f, g)
    df, dg = dc.conv_complex_nd_adjoint(dev(w, dtype), dev(f, dtype), dev(g, dtype))
    N = np.prod([2 * m for m in shape])
    check_parity(df.cpu().numpy(), rdf, dtype, N, norm_scale(w, g))
    check_parity(dg.cpu().numpy(), rdg, dtype, N, norm_scale(w, f))


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
    W = symmetrize_upstream(w)
    check_parity(df.cpu().numpy(), rdf, dtype, N, hermitian_scale(W, g))
    check_parity(dg.cpu().numpy(), rdg, dtype, N, hermitian_scale(W, f))


# --- benchmark shapes -----------------------------------------------------------

def test_hermitian_2d_1024(dc):
    ms = (1024, 1024)
    shape = synthetic.hermitian_shape(ms)
    f = synthetic.hermitian_spectrum(shape, 1.5, 1011)
    g = synthetic.hermitian_spectrum(shape, 1.5, 1012)
    h = dc.conv_hermitian_nd(dev(f, torch.complex64), dev(g, torch.complex64)).cpu().numpy()
    check_parity(h, oracle.padded_hermitian(f, g), torch.complex64, 9 * 1024 * 1024, hermitian_scale(f, g))


def test_complex_2d_2048(dc):
    f = synthetic.uniform_complex((2048, 2048), 1013)
    g = synthetic.uniform_complex((2048, 2048), 1014)
    h = dc.conv_complex_nd(dev(f, torch.complex64), dev(g, torch.complex64)).cpu().numpy()
    check_parity(h, oracle.padded_complex(f, g), torch.complex64, 4 * 2048 * 2048, norm_scale(f, g))


def test_hermitian_3d_256_full(dc):
    """The 3D benchmark shape (511 x 511 x 256, complex64 data, FP64 tables),
    forward, against the explicitly padded FP64 oracle (a 768^3 grid) over
    every output; the call runs the default chunking (several chunks of
    x-slabs with a partial last one)."""
    from paper_1008_1366_gb300 import api
    ms = (256, 256, 256)
    spc, nch = api.chunking(api.KIND_HERMITIAN, ms, api.C64, api.workspace_size(api.KIND_HERMITIAN, ms, api.C64))
    assert nch >= 2 and (3 * 256) % spc != 0, (spc, nch)
    shape = synthetic.hermitian_shape(ms)
    f = synthetic.hermitian_spectrum(shape, 11 / 6, 1015)
    g = synthetic.hermitian_spectrum(shape, 11 / 6, 1016)
    h = dc.conv_hermitian_nd(dev(f, torch.complex64), dev(g, torch.complex64)).cpu().numpy()
    ref = oracle.padded_hermitian(f, g)
    check_parity(h, ref, torch.complex64, 27 * 256 ** 3, hermitian_scale(f, g))


# --- 3D chunks of x-slabs ---------------------------------------------------------
# A 3D call runs its x-level residue slabs (q m_x of them) through the (y, z)
# work arrays a chunk at a time; the chunk follows the workspace.  These
# shapes get a workspace of `spc` slabs, so every call runs at least three
# full chunks and a partial last one.  Last axes 8 and 10 use the
# runtime-shaped row kernel, 64 and 96 the fixed-shape engine.

CHUNK_H = [((8, 6, 8), 7), ((6, 4, 64), 4), ((5, 3, 96), 4), ((6, 5, 10), 5)]
CHUNK_C = [((8, 6, 8), 5), ((8, 4, 64), 5), ((10, 3, 96), 6)]


def _chunks(dc, kind, dims, dtype, spc):
    from paper_1008_1366_gb300 import api
    code = api.dtype_code(torch.empty(0, dtype=dtype))
    ws = api.workspace_size_slabs(kind, dims, code, spc)
    assert ws < api.workspace_size(kind, dims, code)
    got_spc, n = api.chunking(kind, dims, code, ws)
    q = 3 if kind in (api.KIND_HERMITIAN, api.KIND_HERMITIAN_ADJOINT) else 2
    assert got_spc == spc and n == -(-q * dims[0] // spc), (got_spc, n)
    assert n >= 4 and (q * dims[0]) % spc != 0   # at least three full chunks and a partial one
    return n


@pytest.mark.parametrize("ms,spc", CHUNK_H)
@pytest.mark.parametrize("dtype", DT)
def test_hermitian_3d_chunked(dc, ms, spc, dtype):
    from paper_1008_1366_gb300 import api
    _chunks(dc, api.KIND_HERMITIAN, ms, dtype, spc)
    shape = synthetic.hermitian_shape(ms)
    f = synthetic.hermitian_spectrum(shape, 11 / 6, 61)
    g = synthetic.hermitian_spectrum(shape, 11 / 6, 62)
    h = dc.conv_hermitian_nd(dev(f, dtype), dev(g, dtype), slabs_per_chunk=spc).cpu().numpy()
    check_parity(h, oracle.padded_hermitian(f, g), dtype, np.prod([3 * m for m in ms]), hermitian_scale(f, g))
    # the default chunking gives the same outputs to rounding
    h1 = dc.conv_hermitian_nd(dev(f, dtype), dev(g, dtype)).cpu().numpy()
    assert rel_l2(h1, h) <= (1e-15 if dtype == torch.complex128 else 1e-7)


@pytest.mark.parametrize("ms,spc", CHUNK_C)
@pytest.mark.parametrize("dtype", DT)
def test_complex_3d_chunked(dc, ms, spc, dtype):
    from paper_1008_1366_gb300 import api
    _chunks(dc, api.KIND_COMPLEX, ms, dtype, spc)
    f = synthetic.uniform_complex(ms, 63)
    g = synthetic.uniform_complex(ms, 64)
    h = dc.conv_complex_nd(dev(f, dtype), dev(g, dtype), slabs_per_chunk=spc).cpu().numpy()
    check_parity(h, oracle.padded_complex(f, g), dtype, np.prod([2 * m for m in ms]), norm_scale(f, g))


@pytest.mark.parametrize("ms,spc", CHUNK_H)
@pytest.mark.parametrize("dtype", DT)
def test_hermitian_3d_adjoint_chunked(dc, ms, spc, dtype):
    from paper_1008_1366_gb300 import api
    _chunks(dc, api.KIND_HERMITIAN_ADJOINT, ms, dtype, spc)
    shape = synthetic.hermitian_shape(ms)
    f = synthetic.hermitian_spectrum(shape, 11 / 6, 65)
    g = synthetic.hermitian_spectrum(shape, 11 / 6, 66)
    w = synthetic.uniform_complex(shape, 67)
    rdf, rdg = oracle.adjoint_hermitian(w, f, g)
    df, dg = dc.conv_hermitian_nd_adjoint(dev(w, dtype), dev(f, dtype), dev(g, dtype), slabs_per_chunk=spc)
    N = np.prod([3 * m for m in ms])
    W = symmetrize_upstream(w)
    check_parity(df.cpu().numpy(), rdf, dtype, N, hermitian_scale(W, g))
    check_parity(dg.cpu().numpy(), rdg, dtype, N, hermitian_scale(W, f))


@pytest.mark.parametrize("ms,spc", CHUNK_C)
@pytest.mark.parametrize("dtype", DT)
def test_complex_3d_adjoint_chunked(dc, ms, spc, dtype):
    from paper_1008_1366_gb300 import api
    _chunks(dc, api.KIND_COMPLEX_ADJOINT, ms, dtype, spc)
    w, f, g = (synthetic.uniform_complex(ms, s) for s in (68, 69, 70))
    rdf, rdg = oracle.adjoint_complex(w, f, g, padded=True)
    df, dg = dc.conv_complex_nd_adjoint(dev(w, dtype), dev(f, dtype), dev(g, dtype), slabs_per_chunk=spc)
    N = np.prod([2 * m for m in ms])
    check_parity(df.cpu().numpy(), rdf, dtype, N, norm_scale(w, g))
    check_parity(dg.cpu().numpy(), rdg, dtype, N, norm_scale(w, f))


def test_workspace_below_one_slab_is_refused(dc):
    import ctypes
    from paper_1008_1366_gb300 import _native, api
    dims = (4, 3, 8)
    code = api.C128
    ws1 = api.workspace_size_slabs(api.KIND_HERMITIAN, dims, code, 1)
    assert api.chunking(api.KIND_HERMITIAN, dims, code, ws1 - 256) == (0, 0)
    shape = synthetic.hermitian_shape(dims)
    t = torch.zeros(shape, dtype=torch.complex128, device="cuda")
    work = torch.zeros(ws1, dtype=torch.uint8, device="cuda")
    L = _native.lib()
    vp = lambda x: ctypes.c_void_p(x.data_ptr())
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.dc_conv_hermitian_3d(vp(t), vp(t), vp(t), *dims, code, vp(work), ws1 - 256, s) == 6
    assert L.dc_conv_hermitian_3d(vp(t), vp(t), vp(t), *dims, code, vp(work), ws1, s) == 0
    torch.cuda.synchronize()

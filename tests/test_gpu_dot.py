"""GPU parity of the dot products of two pairs (Sec. 3, 2D pseudospectral
application: the product f * g of arrays of vectors read as
f1 * g1 + f2 * g2, with one forward transform per residue for both pairs)
against the FP64 oracle (oracle.dot_complex / dot_hermitian), through the C
ABI, in 1D, 2D and 3D, both precisions, with both error bars of
conftest.check_parity; and the paper's example, the advective term of the
2D Euler equation."""

import numpy as np
import pytest
import torch

import oracle
from conftest import check_parity, hermitian_scale, norm_scale, rel_l2
from paper_1008_1366_gb300 import synthetic

pytestmark = pytest.mark.gpu

DT = [torch.complex128, torch.complex64]


@pytest.fixture(scope="module")
def dc():
    import paper_1008_1366_gb300 as dc
    return dc


def dev(x, dtype):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


def dot_scale(fs, gs, hermitian):
    sc = hermitian_scale if hermitian else norm_scale
    return sum(sc(f, g) for f, g in zip(fs, gs))


@pytest.mark.parametrize("m", [1, 2, 5, 64, 96, 640, 1024, 4096, 16384, 20480])
@pytest.mark.parametrize("dtype", DT)
def test_complex_dot2_1d(dc, m, dtype):
    fs = [synthetic.uniform_complex(m, 50 + s) for s in (0, 1)]
    gs = [synthetic.uniform_complex(m, 52 + s) for s in (0, 1)]
    h = dc.conv_complex_dot2(dev(fs[0], dtype), dev(gs[0], dtype), dev(fs[1], dtype), dev(gs[1], dtype))
    check_parity(h.cpu().numpy(), oracle.dot_complex(fs, gs), dtype, 2 * m, dot_scale(fs, gs, False))


@pytest.mark.parametrize("m", [1, 2, 5, 9, 64, 96, 640, 1024, 4096, 16384, 20480])
@pytest.mark.parametrize("dtype", DT)
def test_hermitian_dot2_1d(dc, m, dtype):
    fs = [synthetic.hermitian_spectrum((m,), 1.0, 54 + s) for s in (0, 1)]
    gs = [synthetic.hermitian_spectrum((m,), 1.0, 56 + s) for s in (0, 1)]
    h = dc.conv_hermitian_dot2(dev(fs[0], dtype), dev(gs[0], dtype), dev(fs[1], dtype), dev(gs[1], dtype))
    check_parity(h.cpu().numpy(), oracle.dot_hermitian(fs, gs), dtype, 3 * m, dot_scale(fs, gs, True))


# rows of 64 (and 2, 3, 64 in 3D) on the fixed engine's dot-product residues,
# rows of 8192 (a two-level size) and other lengths on the runtime-shaped kernel
@pytest.mark.parametrize("ms", [(1, 1), (3, 4), (8, 8), (16, 12), (64, 64), (9, 15), (2, 3, 4), (4, 4, 6),
                                (3, 8192), (2, 3, 64)])
@pytest.mark.parametrize("dtype", DT)
def test_hermitian_dot2_nd(dc, ms, dtype):
    shape = synthetic.hermitian_shape(ms)
    fs = [synthetic.hermitian_spectrum(shape, 1.5, 58 + s) for s in (0, 1)]
    gs = [synthetic.hermitian_spectrum(shape, 1.5, 60 + s) for s in (0, 1)]
    h = dc.conv_hermitian_dot2(*[dev(x, dtype) for x in (fs[0], gs[0], fs[1], gs[1])])
    check_parity(h.cpu().numpy(), oracle.dot_hermitian(fs, gs), dtype, np.prod([3 * m for m in ms]),
                 dot_scale(fs, gs, True))


@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (8, 8), (32, 48), (4, 6, 5)])
@pytest.mark.parametrize("dtype", DT)
def test_complex_dot2_nd(dc, shape, dtype):
    fs = [synthetic.uniform_complex(shape, 62 + s) for s in (0, 1)]
    gs = [synthetic.uniform_complex(shape, 64 + s) for s in (0, 1)]
    h = dc.conv_complex_dot2(*[dev(x, dtype) for x in (fs[0], gs[0], fs[1], gs[1])])
    check_parity(h.cpu().numpy(), oracle.dot_complex(fs, gs), dtype, np.prod([2 * m for m in shape]),
                 dot_scale(fs, gs, False))


@pytest.mark.parametrize("dtype", DT)
def test_hermitian_dot2_3d_chunked(dc, dtype):
    # 3D: x-slabs in at least three full chunks and a partial one
    ms, spc = (6, 4, 8), 5
    shape = synthetic.hermitian_shape(ms)
    fs = [synthetic.hermitian_spectrum(shape, 11 / 6, 66 + s) for s in (0, 1)]
    gs = [synthetic.hermitian_spectrum(shape, 11 / 6, 68 + s) for s in (0, 1)]
    h = dc.conv_hermitian_dot2(*[dev(x, dtype) for x in (fs[0], gs[0], fs[1], gs[1])], slabs_per_chunk=spc)
    check_parity(h.cpu().numpy(), oracle.padded_hermitian(fs[0], gs[0]) + oracle.padded_hermitian(fs[1], gs[1]),
                 dtype, np.prod([3 * m for m in ms]), dot_scale(fs, gs, True))


def euler_inputs(ms, seed):
    """The paper's call for the 2D Euler advective term: f = (i kx w, i ky w)
    (grad w), g = (i ky w / k^2, -i kx w / k^2) (the velocity); the zero mode
    of w / k^2 is taken as 0."""
    shape = synthetic.hermitian_shape(ms)
    w = synthetic.hermitian_spectrum(shape, 1.5, seed)
    mx = ms[0]
    kx = (np.arange(shape[0]) - (mx - 1))[:, None] * np.ones((1, shape[1]))
    ky = np.ones((shape[0], 1)) * np.arange(shape[1])[None, :]
    k2 = kx ** 2 + ky ** 2
    inv = np.where(k2 > 0, 1.0 / np.where(k2 > 0, k2, 1.0), 0.0)
    return [1j * kx * w, 1j * ky * w], [1j * ky * w * inv, -1j * kx * w * inv]


@pytest.mark.parametrize("ms,dtype", [((32, 32), torch.complex128), ((32, 32), torch.complex64),
                                      ((1024, 1024), torch.complex64)])
def test_euler_advective_term(dc, ms, dtype):
    fs, gs = euler_inputs(ms, 70)
    h = dc.conv_hermitian_dot2(*[dev(x, dtype) for x in (fs[0], gs[0], fs[1], gs[1])]).cpu().numpy()
    ref = oracle.dot_hermitian(fs, gs)
    check_parity(h, ref, dtype, 9 * ms[0] * ms[1], dot_scale(fs, gs, True))
    # the same as the two convolutions of the separate calls, added
    h2 = sum(dc.conv_hermitian_nd(dev(f, dtype), dev(g, dtype)).cpu().numpy() for f, g in zip(fs, gs))
    assert rel_l2(h, h2) <= (1e-13 if dtype == torch.complex128 else 5e-6)


def test_dot2_in_place_and_argument_checks(dc):
    import ctypes
    from paper_1008_1366_gb300 import _native, api
    m = 1024
    fs = [synthetic.uniform_complex(m, 71 + s) for s in (0, 1)]
    gs = [synthetic.uniform_complex(m, 73 + s) for s in (0, 1)]
    ref = oracle.dot_complex(fs, gs)
    ts = [dev(x, torch.complex128) for x in (fs[0], gs[0], fs[1], gs[1])]
    L = _native.lib()
    ws = api.workspace_size(api.KIND_COMPLEX_DOT2, [m], api.C128)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    d = (ctypes.c_int64 * 1)(m)
    # in place: h is f1
    assert L.dc_conv_complex_dot2(1, d, *[vp(t) for t in ts], vp(ts[0]), 1, vp(work), ws, s) == 0
    torch.cuda.synchronize()
    check_parity(ts[0].cpu().numpy(), ref, torch.complex128, 2 * m, dot_scale(fs, gs, False))
    assert L.dc_conv_complex_dot2(4, d, *[vp(t) for t in ts], vp(ts[0]), 1, vp(work), ws, s) == 1
    assert L.dc_conv_complex_dot2(1, d, *[vp(t) for t in ts[:3]], None, vp(ts[0]), 1, vp(work), ws, s) == 1
    assert L.dc_conv_complex_dot2(1, d, *[vp(t) for t in ts], vp(ts[0]), 1, vp(work), 16, s) == 6

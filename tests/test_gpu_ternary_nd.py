"""GPU parity of the 2D and 3D centered Hermitian ternary convolutions
(Sec. 4: Function tconv2, the outer axes padded implicitly to N = 4m,
Eqs. (fft0tbackward)-(fft0tforward): as two residues of 2m-point
sub-transforms, or, where every outer length is a power of two from 64 to
4096, as four m-point residues; the last axis by the 1D ternary rows of
Sec. 4.2) against the FP64 oracle, every output, both error bars of
conftest.check_parity, both precisions; the paper's 4096 x 4096 shape
(Fig. 9) in FP32."""

import numpy as np
import pytest
import torch

import oracle
from conftest import check_parity, hermitian_scale

pytestmark = pytest.mark.gpu

from paper_1008_1366_gb300 import synthetic  # noqa: E402

DT = [torch.complex128, torch.complex64]


@pytest.fixture(scope="module")
def dc():
    import paper_1008_1366_gb300 as dc
    return dc


def dev(x, dtype):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


def inputs(ms, seed, alpha):
    shape = synthetic.hermitian_shape(ms)
    return [synthetic.hermitian_spectrum(shape, alpha, seed + s) for s in range(3)]


# (64, 64), (128, 96), (256, 40), (512, 3), (2048, 5): four m-point residues on the x axis
T2 = [(1, 1), (2, 2), (3, 4), (4, 4), (8, 6), (5, 9), (16, 16), (32, 24), (64, 64), (128, 96), (9, 15),
      (256, 40), (512, 3), (2048, 5)]


@pytest.mark.parametrize("ms", T2)
@pytest.mark.parametrize("dtype", DT)
def test_ternary_2d(dc, ms, dtype):
    f, g, e = inputs(ms, 80, 1.5)
    h = dc.conv_ternary_hermitian_nd(dev(f, dtype), dev(g, dtype), dev(e, dtype)).cpu().numpy()
    check_parity(h, oracle.conv_ternary_hermitian(f, g, e), dtype, np.prod([4 * m for m in ms]),
                 hermitian_scale(f, g, e))


# (64, 64, 8), (64, 128, 6): four m-point residues on both outer axes,
# the second in chunks of 37 slabs (the last one partial); (8, 8, 64),
# (64, 64, 64): rows of a one-level size of the set on the fixed engine's
# four-residue ternary kind (in 2D: (64, 64), (128, 96), 4096 x 4096)
@pytest.mark.parametrize("ms,spc", [((2, 2, 2), None), ((3, 4, 5), None), ((4, 4, 4), 3), ((5, 3, 8), 7),
                                    ((8, 8, 16), None), ((64, 64, 8), None), ((64, 128, 6), 37),
                                    ((8, 8, 64), None), ((64, 64, 64), 50)])
@pytest.mark.parametrize("dtype", DT)
def test_ternary_3d(dc, ms, spc, dtype):
    f, g, e = inputs(ms, 84, 11 / 6)
    h = dc.conv_ternary_hermitian_nd(dev(f, dtype), dev(g, dtype), dev(e, dtype), slabs_per_chunk=spc).cpu().numpy()
    check_parity(h, oracle.padded_ternary_hermitian(f, g, e), dtype, np.prod([4 * m for m in ms]),
                 hermitian_scale(f, g, e))


def test_ternary_2d_projects_raw_inputs(dc):
    ms = (4, 6)
    shape = synthetic.hermitian_shape(ms)
    f, g, e = (synthetic.uniform_complex(shape, s) for s in (87, 88, 89))
    h = dc.conv_ternary_hermitian_nd(*[dev(x, torch.complex128) for x in (f, g, e)]).cpu().numpy()
    check_parity(h, oracle.conv_ternary_hermitian(f, g, e), torch.complex128, 16 * 4 * 6, hermitian_scale(f, g, e))


def test_ternary_2d_in_place(dc):
    ms = (16, 12)
    f, g, e = inputs(ms, 90, 1.5)
    ref = oracle.conv_ternary_hermitian(f, g, e)
    for target in range(3):
        ts = [dev(x, torch.complex128) for x in (f, g, e)]
        from paper_1008_1366_gb300 import api
        import ctypes
        dims = (16, 12)
        ws = api.workspace_size(api.KIND_TERNARY, dims, api.C128)
        work = torch.empty(ws, dtype=torch.uint8, device="cuda")
        vp = lambda t: ctypes.c_void_p(t.data_ptr())
        st = api._native.lib().dc_conv_ternary_hermitian_2d(*[vp(t) for t in ts], vp(ts[target]), *dims, api.C128,
                                                              vp(work), ws,
                                                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0
        torch.cuda.synchronize()
        check_parity(ts[target].cpu().numpy(), ref, torch.complex128, 16 * 16 * 12, hermitian_scale(f, g, e))


def test_ternary_2d_4096(dc):
    """The shape of the paper's 2D ternary timings (Fig. 9), mx = my = 4096,
    complex64 data, against the explicitly padded FP64 oracle (a 16384^2
    grid) over every output."""
    ms = (4096, 4096)
    f, g, e = inputs(ms, 1030, 1.5)
    h = dc.conv_ternary_hermitian_nd(*[dev(x, torch.complex64) for x in (f, g, e)]).cpu().numpy()
    ref = oracle.padded_ternary_hermitian(f, g, e)
    check_parity(h, ref, torch.complex64, 16 * 4096 * 4096, hermitian_scale(f, g, e))

"""GPU parity of the 1D kernels against the FP64 oracle, through the C ABI.

Sizes span several tiles, both kernel levels (shared-memory resident and
two-level through scratch), every radix (2, 3, 4, 5, 8, 16), ragged small
cases and the degenerate m = 1.  Bars: relative L2 <= 1e-12 for the FP64
path, <= 5e-7 log2(N) for FP32 with N the implicit padded size, and every
output within the pointwise bar of conftest.check_parity."""

import numpy as np
import pytest
import torch

import oracle
from oracle.adjoint import symmetrize_upstream
from conftest import FP64_TOL, check_parity, fp32_tol, hermitian_scale, norm_scale, rel_l2
from paper_1008_1366_gb300 import synthetic

pytestmark = pytest.mark.gpu

SMALL = [1, 2, 3, 4, 5, 6, 8, 10, 12, 16, 20, 24, 32, 40, 48, 64, 80, 96, 160, 192, 256, 320, 384, 640]
LARGE = [1024, 1536, 2560, 4096, 6144, 8192, 10240, 12288, 16384, 20480, 24576, 32768, 40960, 49152, 65536]
DTYPES = [(torch.complex128, None), (torch.complex64, "fp32")]


@pytest.fixture(scope="module")
def dc():
    import paper_1008_1366_gb300 as dc
    return dc


def tol_for(dtype, N):
    return FP64_TOL if dtype == torch.complex128 else fp32_tol(N)


def to_dev(x, dtype):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


@pytest.mark.parametrize("m", SMALL + LARGE)
@pytest.mark.parametrize("dtype", [d for d, _ in DTYPES])
def test_complex_1d(dc, m, dtype):
    f = synthetic.uniform_complex(m, 100 + m)
    g = synthetic.uniform_complex(m, 200 + m)
    ref = oracle.conv_complex(f, g)
    h = dc.conv_complex_1d(to_dev(f, dtype), to_dev(g, dtype)).cpu().numpy()
    check_parity(h, ref, dtype, 2 * m, norm_scale(f, g))


def test_complex_1d_paper_closed_form(dc):
    # the paper's accuracy test of Sec. 2.1 at m = 1024 in FP64
    m = 1024
    k = np.arange(m)
    F, G = np.sqrt(3) + 1j * np.sqrt(7), np.sqrt(5) + 1j * np.sqrt(11)
    f, g = F * np.exp(1j * k), G * np.exp(1j * k)
    H = F * G * (k + 1) * np.exp(1j * k)
    h = dc.conv_complex_1d(to_dev(f, torch.complex128), to_dev(g, torch.complex128)).cpu().numpy()
    assert rel_l2(h, H) <= 1e-13


def test_complex_1d_in_place(dc):
    m = 4096
    f = synthetic.uniform_complex(m, 1)
    g = synthetic.uniform_complex(m, 2)
    tf = to_dev(f, torch.complex128)
    out = dc.conv_complex_1d(tf, to_dev(g, torch.complex128), out=tf)
    assert out.data_ptr() == tf.data_ptr()
    check_parity(tf.cpu().numpy(), oracle.conv_complex(f, g), torch.complex128, 2 * m, norm_scale(f, g))


# 8192 and up (in the size set): the fixed-shape engine's two-level passes
HERM = [1, 2, 4, 6, 8, 10, 12, 16, 20, 24, 40, 48, 64, 96, 160, 256, 1024, 3072, 5120, 8192, 10240, 12288, 16384,
        20480, 24576, 32768, 40960, 49152, 65536]


@pytest.mark.parametrize("m", HERM)
@pytest.mark.parametrize("dtype", [d for d, _ in DTYPES])
def test_hermitian_1d(dc, m, dtype):
    f = synthetic.hermitian_spectrum((m,), 1.0, 300 + m)
    g = synthetic.hermitian_spectrum((m,), 1.0, 400 + m)
    ref = oracle.conv_hermitian(f, g)
    h = dc.conv_hermitian_1d(to_dev(f, dtype), to_dev(g, dtype)).cpu().numpy()
    check_parity(h, ref, dtype, 3 * m, hermitian_scale(f, g))


@pytest.mark.parametrize("m", [96, 4096, 8192, 20480, 65536])
def test_hermitian_1d_flat_spectrum_fp32(dc, m):
    # unit amplitude at every wavenumber: all outputs are of one magnitude,
    # so the global bar also sees an error confined to the high wavenumbers
    f = synthetic.hermitian_spectrum((m,), 0.0, 350 + m)
    g = synthetic.hermitian_spectrum((m,), 0.0, 450 + m)
    ref = oracle.conv_hermitian(f, g)
    h = dc.conv_hermitian_1d(to_dev(f, torch.complex64), to_dev(g, torch.complex64)).cpu().numpy()
    check_parity(h, ref, torch.complex64, 3 * m, hermitian_scale(f, g))


@pytest.mark.parametrize("m", [256, 16384])
def test_hermitian_1d_projection_of_raw_input(dc, m):
    # a non-real f_0 is projected to Re f_0, like the oracle
    f = synthetic.uniform_complex(m, 5)
    g = synthetic.uniform_complex(m, 6)
    h = dc.conv_hermitian_1d(to_dev(f, torch.complex128), to_dev(g, torch.complex128)).cpu().numpy()
    check_parity(h, oracle.conv_hermitian(f, g), torch.complex128, 3 * m, hermitian_scale(f, g))


@pytest.mark.parametrize("m", [1024, 24576])
@pytest.mark.parametrize("dtype", [d for d, _ in DTYPES])
def test_hermitian_1d_in_place(dc, m, dtype):
    # h may be f or g: every read of the inputs precedes the first write of h
    f = synthetic.hermitian_spectrum((m,), 1.0, 31)
    g = synthetic.hermitian_spectrum((m,), 1.0, 32)
    ref = oracle.conv_hermitian(f, g)
    for target in ("f", "g"):
        tf, tg = to_dev(f, dtype), to_dev(g, dtype)
        out = tf if target == "f" else tg
        dc.conv_hermitian_1d(tf, tg, out=out)
        check_parity(out.cpu().numpy(), ref, dtype, 3 * m, hermitian_scale(f, g))


@pytest.mark.parametrize("m", [4096, 32768])
def test_hermitian_1d_paper_closed_form(dc, m):
    k = np.arange(m)
    f, g = np.sqrt(3) * np.exp(1j * k), np.sqrt(5) * np.exp(1j * k)
    H = np.sqrt(15) * (2 * m - 1 - k) * np.exp(1j * k)
    h = dc.conv_hermitian_1d(to_dev(f, torch.complex128), to_dev(g, torch.complex128)).cpu().numpy()
    assert rel_l2(h, H) <= 1e-13


# 4096 and up with 2m in the size set: the fixed-shape engine's two-level
# passes over the 2m-point sub-transforms
TERN = [1, 2, 3, 4, 5, 8, 12, 16, 20, 64, 96, 160, 1024, 2048, 4096, 5120, 6144, 8192, 10240, 12288, 16384,
        20480, 24576, 32768]


@pytest.mark.parametrize("m", TERN)
@pytest.mark.parametrize("dtype", [d for d, _ in DTYPES])
def test_ternary_1d(dc, m, dtype):
    f, g, e = (synthetic.hermitian_spectrum((m,), 1.0, s + m) for s in (500, 600, 700))
    ref = oracle.conv_ternary_hermitian(f, g, e)
    h = dc.conv_ternary_hermitian_1d(to_dev(f, dtype), to_dev(g, dtype), to_dev(e, dtype)).cpu().numpy()
    check_parity(h, ref, dtype, 4 * m, hermitian_scale(f, g, e))


@pytest.mark.parametrize("m", [160, 16384])
def test_ternary_1d_projection_and_in_place(dc, m):
    # raw inputs (non-real U_0 projected to its real part, like the oracle);
    # the output may be any of the three inputs
    f, g, e = (synthetic.uniform_complex(m, s) for s in (41, 42, 43))
    ref = oracle.conv_ternary_hermitian(f, g, e)
    dtype = torch.complex128
    S = hermitian_scale(f, g, e)
    check_parity(dc.conv_ternary_hermitian_1d(to_dev(f, dtype), to_dev(g, dtype), to_dev(e, dtype)).cpu().numpy(),
                 ref, dtype, 4 * m, S)
    for target in range(3):
        ts = [to_dev(x, dtype) for x in (f, g, e)]
        dc.conv_ternary_hermitian_1d(*ts, out=ts[target])
        check_parity(ts[target].cpu().numpy(), ref, dtype, 4 * m, S)


@pytest.mark.parametrize("m", [1, 3, 16, 80, 1024, 12288, 32768])
@pytest.mark.parametrize("dtype", [d for d, _ in DTYPES])
def test_complex_1d_adjoint(dc, m, dtype):
    w, f, g = (synthetic.uniform_complex(m, s + m) for s in (1, 2, 3))
    rdf, rdg = oracle.adjoint_complex(w, f, g)
    df, dg = dc.conv_complex_1d_adjoint(to_dev(w, dtype), to_dev(f, dtype), to_dev(g, dtype))
    check_parity(df.cpu().numpy(), rdf, dtype, 2 * m, norm_scale(w, g))
    check_parity(dg.cpu().numpy(), rdg, dtype, 2 * m, norm_scale(w, f))


@pytest.mark.parametrize("m", [1, 2, 8, 96, 1024, 16384])
@pytest.mark.parametrize("dtype", [d for d, _ in DTYPES])
def test_hermitian_1d_adjoint(dc, m, dtype):
    f = synthetic.hermitian_spectrum((m,), 1.0, 7)
    g = synthetic.hermitian_spectrum((m,), 1.0, 8)
    w = synthetic.uniform_complex(m, 9)
    rdf, rdg = oracle.adjoint_hermitian(w, f, g)
    df, dg = dc.conv_hermitian_1d_adjoint(to_dev(w, dtype), to_dev(f, dtype), to_dev(g, dtype))
    W = symmetrize_upstream(w)
    check_parity(df.cpu().numpy(), rdf, dtype, 3 * m, hermitian_scale(W, g))
    check_parity(dg.cpu().numpy(), rdg, dtype, 3 * m, hermitian_scale(W, f))


@pytest.mark.parametrize("dtype", [d for d, _ in DTYPES])
def test_batched_mixed_sizes(dc, dtype):
    sizes = [64, 80, 96, 1, 7 * 0 + 5, 128, 3072, 65536, 10240, 160, 64, 64, 96, 20480, 8192, 40960]
    f, g, off = synthetic.batched_inputs(sizes, 11)
    plan = dc.BatchedPlan(sizes, dtype=dtype)
    assert plan.launches == 1
    h = plan(to_dev(f, dtype), to_dev(g, dtype)).cpu().numpy()
    for i, m in enumerate(sizes):
        a, b = off[i], off[i + 1]
        ref = oracle.conv_complex(f[a:b], g[a:b])
        check_parity(h[a:b], ref, dtype, 2 * m, norm_scale(f[a:b], g[a:b]), what=f"instance {i} m={m}")


def test_batched_one_per_launch_matches(dc):
    sizes = [64, 1024, 96, 16384, 80]
    f, g, off = synthetic.batched_inputs(sizes, 12)
    a = dc.BatchedPlan(sizes, dtype=torch.complex128)
    b = dc.BatchedPlan(sizes, dtype=torch.complex128, flags=4)
    assert b.launches == len(sizes)
    ha = a(to_dev(f, torch.complex128), to_dev(g, torch.complex128)).cpu().numpy()
    hb = b(to_dev(f, torch.complex128), to_dev(g, torch.complex128)).cpu().numpy()
    assert rel_l2(hb, ha) <= 1e-14


def test_status_codes(dc):
    import ctypes
    from paper_1008_1366_gb300 import _native
    L = _native.lib()
    t = torch.zeros(64, dtype=torch.complex64, device="cuda")
    w = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    vp = lambda x: ctypes.c_void_p(x.data_ptr())
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.dc_conv_complex_1d(vp(t), vp(t), vp(t), 7, 0, vp(w), w.numel(), s) == 2     # 7 unsupported
    assert L.dc_conv_complex_1d(vp(t), vp(t), vp(t), 64, 0, vp(w), 16, s) == 6          # workspace too small
    assert L.dc_conv_complex_1d(vp(t), vp(t), vp(t), 64, 0, ctypes.c_void_p(w.data_ptr() + 8), w.numel() - 8, s) == 3
    assert L.dc_conv_hermitian_1d(vp(t), vp(t), vp(t), 14, 0, vp(w), w.numel(), s) == 2  # 14 = 2*7
    h = dc.conv_complex_1d(t, t)
    assert dc.read_status(torch.zeros(256, dtype=torch.uint8, device="cuda")) == (0, 0)
    torch.cuda.synchronize()
    assert h.abs().max().item() == 0

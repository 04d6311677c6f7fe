"""torch.autograd.Function wrappers: forward is the dealiased convolution,
backward the library's adjoint kernels (correlations with the conjugate
partner, computed by the same residue machinery).

PyTorch's complex-gradient convention applies: for a real loss L the
gradient of a complex tensor z is dL/dRe z + i dL/dIm z, so for
L = Re sum conj(w) h the incoming grad_output is w itself and the returned
gradients are exactly what the adjoint entry points compute.
"""

import torch

from . import api


def _conv(kind, f, g):
    if f.dim() == 1:
        return api.conv_complex_1d(f, g) if kind == "complex" else api.conv_hermitian_1d(f, g)
    return api.conv_complex_nd(f, g) if kind == "complex" else api.conv_hermitian_nd(f, g)


def _adjoint(kind, w, f, g):
    if f.dim() == 1:
        fn = api.conv_complex_1d_adjoint if kind == "complex" else api.conv_hermitian_1d_adjoint
    else:
        fn = api.conv_complex_nd_adjoint if kind == "complex" else api.conv_hermitian_nd_adjoint
    return fn(w, f, g)


class _Conv(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kind, f, g):
        f = f.contiguous()
        g = g.contiguous()
        ctx.kind = kind
        ctx.save_for_backward(f, g)
        return _conv(kind, f, g)

    @staticmethod
    def backward(ctx, w):
        f, g = ctx.saved_tensors
        df, dg = _adjoint(ctx.kind, w.contiguous(), f, g)
        return None, (df if ctx.needs_input_grad[1] else None), (dg if ctx.needs_input_grad[2] else None)


def conv_complex(f, g):
    """Differentiable complex dealiased convolution (1D, 2D or 3D)."""
    return _Conv.apply("complex", f, g)


def conv_hermitian(f, g):
    """Differentiable centered Hermitian dealiased convolution (1D, 2D or 3D)."""
    return _Conv.apply("hermitian", f, g)

"""GB300 (sm_103a) implicitly dealiased convolutions (Bowman & Roberts 2011).

The compute path is libdealias.so (hand-written CUDA, C ABI in
include/dealias.h); this package is its thin PyTorch binding.
"""

from .api import (  # noqa: F401
    BatchedPlan,
    chunking,
    DealiasError,
    conv_complex_1d,
    conv_complex_1d_adjoint,
    conv_complex_1d_full,
    conv_complex_1d_pq,
    conv_complex_dot2,
    conv_complex_nd,
    conv_complex_nd_adjoint,
    conv_hermitian_nd,
    conv_hermitian_nd_adjoint,
    conv_hermitian_1d,
    conv_hermitian_1d_adjoint,
    conv_hermitian_dot2,
    conv_ternary_hermitian_1d,
    conv_ternary_hermitian_nd,
    partition_lpt,
    prepare,
    read_status,
    read_trace,
    shard,
    workspace_size,
    workspace_size_slabs,
)

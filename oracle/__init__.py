"""FP64 CPU oracle for the dealiased convolutions of Bowman & Roberts,
"Efficient Dealiased Convolutions without Padding" (SIAM J. Sci. Comput. 2011).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library, its
C ABI and the Python binding in ``paper_1008_1366_gb300``) imports, links or
executes anything in this package.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py`` use it.

The oracle shares no code with the GPU path.  It does not implement the
implicit (residue sub-transform) method at all: it computes the plain
definition of each convolution that the method reproduces up to rounding,

  * ``direct_*``  -- the defining sums written out (small sizes), and
  * ``padded_*``  -- the conventional explicitly zero-padded FFT convolution the
                     paper starts from (Sec. 1), with numpy's FFT as a library
                     step (large sizes), and
  * ``*_at``      -- the defining sums at selected output indices (spot checks
                     at sizes where the full oracle is too slow).

All arithmetic is complex128 / float64.  Pins tying these functions to facts
outside themselves (brute force, the paper's closed forms, polynomial
identities, symmetries, separability, finite differences) live in
``tests/test_oracle_*.py``.  Every function is pinned; none is "parity
unpinned".
"""

from .conv import (  # noqa: F401
    project_hermitian,
    hermitian_extend,
    direct_complex,
    padded_complex,
    direct_hermitian,
    padded_hermitian,
    direct_ternary_hermitian,
    padded_ternary_hermitian,
    complex_at,
    hermitian_at,
    conv_complex,
    conv_hermitian,
    conv_ternary_hermitian,
    direct_complex_pq,
    padded_complex_pq,
    dot_complex,
    dot_hermitian,
)
from .adjoint import (  # noqa: F401
    loss,
    grad_by_linearity,
    adjoint_complex,
    adjoint_hermitian,
    adjoint_ternary_hermitian,
)

"""PyTorch-facing binding of the C ABI (argument marshalling only).

Every function takes CUDA tensors (complex64 -> FP32 path, complex128 -> FP64
path), checks shapes on the host, allocates the output and workspace with
PyTorch's allocator, and calls the matching ``dc_*`` entry point of
libdealias.so on the current stream.  All arithmetic runs in the library's
kernels.
"""

import ctypes

import torch

from . import _native

C64, C128 = 0, 1
(KIND_COMPLEX, KIND_HERMITIAN, KIND_TERNARY, KIND_COMPLEX_ADJOINT, KIND_HERMITIAN_ADJOINT,
 KIND_COMPLEX_DOT2, KIND_HERMITIAN_DOT2) = range(7)
PLAN_AUTOTUNE = 1
PLAN_ONE_PER_LAUNCH = 4


class DealiasError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(msg)
        self.status = status


def check(status, what):
    if status != 0:
        L = _native.lib()
        msg = L.dc_status_string(status).decode()
        if status == 4:
            msg += f" (cudaError {L.dc_last_cuda_error()})"
        raise DealiasError(status, f"{what}: {msg}")


def dtype_code(t):
    if t.dtype == torch.complex64:
        return C64
    if t.dtype == torch.complex128:
        return C128
    raise TypeError(f"expected complex64 or complex128, got {t.dtype}")


def _stream(t):
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _vp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _inputs(*ts):
    ref = ts[0]
    if not ref.is_cuda:
        raise ValueError("inputs must be CUDA tensors (no CPU path exists)")
    for t in ts:
        if t.device != ref.device or t.dtype != ref.dtype or t.shape != ref.shape:
            raise ValueError("inputs must share device, dtype and shape")
        if not t.is_contiguous():
            raise ValueError("inputs must be contiguous")
    return dtype_code(ref)


def workspace_size(kind, dims, dtype):
    d = (ctypes.c_int64 * len(dims))(*[int(x) for x in dims])
    out = ctypes.c_size_t(0)
    check(_native.lib().dc_workspace_size(kind, len(dims), d, dtype, ctypes.byref(out)), "dc_workspace_size")
    return int(out.value)


def workspace_size_slabs(kind, dims, dtype, slabs_per_chunk):
    """Workspace of a 3D call whose chunks hold at most this many x-slabs
    (dc_workspace_size_slabs)."""
    d = (ctypes.c_int64 * len(dims))(*[int(x) for x in dims])
    out = ctypes.c_size_t(0)
    check(_native.lib().dc_workspace_size_slabs(kind, len(dims), d, dtype, int(slabs_per_chunk),
                                                ctypes.byref(out)), "dc_workspace_size_slabs")
    return int(out.value)


def chunking(kind, dims, dtype, work_bytes):
    """(slabs per chunk, chunks) of a multi-D call with this workspace (dc_chunking)."""
    d = (ctypes.c_int64 * len(dims))(*[int(x) for x in dims])
    s, c = ctypes.c_int64(0), ctypes.c_int64(0)
    check(_native.lib().dc_chunking(kind, len(dims), d, dtype, int(work_bytes), ctypes.byref(s), ctypes.byref(c)),
          "dc_chunking")
    return int(s.value), int(c.value)


def prepare(kind, dims, dtype):
    d = (ctypes.c_int64 * len(dims))(*[int(x) for x in dims])
    check(_native.lib().dc_prepare(kind, len(dims), d, dtype), "dc_prepare")


def _work(nbytes, device):
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def read_status(work):
    st, det = ctypes.c_int32(0), ctypes.c_int32(0)
    check(_native.lib().dc_read_status(_vp(work), _stream(work), ctypes.byref(st), ctypes.byref(det)),
          "dc_read_status")
    return st.value, det.value


def read_trace(work):
    """Trace counters of the last fixed-engine launch on `work`
    (dc_read_trace): waits, and SM cycles / task counts per task type."""
    out = (ctypes.c_uint64 * 12)()
    check(_native.lib().dc_read_trace(_vp(work), _stream(work), out), "dc_read_trace")
    names = ("L1", "A", "B", "C")
    return {"waited": out[0], "wait_cycles": out[1],
            "cycles": dict(zip(names, out[2:6])), "tasks": dict(zip(names, out[6:10])),
            "handover_cycles": out[10], "table_cycles": out[11]}


def _run_1d(name, kind, ins, nout, out):
    dt = _inputs(*ins)
    if ins[0].dim() != 1:
        raise ValueError(f"{name}: expected 1D tensors")
    m = ins[0].shape[0]
    outs = list(out) if out is not None else [torch.empty_like(ins[0]) for _ in range(nout)]
    ws = workspace_size(kind, [m], dt)
    work = _work(ws, ins[0].device)
    fn = getattr(_native.lib(), name)
    args = [_vp(t) for t in ins] + [_vp(t) for t in outs]
    check(fn(*args, m, dt, _vp(work), ws, _stream(ins[0])), name)
    return outs[0] if nout == 1 else tuple(outs)


def conv_complex_1d(f, g, out=None):
    """h_k = sum_{p<=k} f_p g_{k-p}, k < m (dc_conv_complex_1d)."""
    return _run_1d("dc_conv_complex_1d", KIND_COMPLEX, [f, g], 1, None if out is None else [out])


def conv_complex_1d_pq(f, g, m, p, q, nout=None):
    """General implicit padding (dc_conv_complex_1d_pq): f, g hold p m values,
    zero padded to q m; returns the nout first outputs of the padded cyclic
    convolution (default: the full linear convolution, 2pm - 1 outputs, when
    q >= 2p, else all q m)."""
    dt = _inputs(f, g)
    if f.dim() != 1 or f.shape[0] != p * m:
        raise ValueError("inputs must be 1D of length p * m")
    nout = int(nout) if nout is not None else (2 * p * m - 1 if q >= 2 * p else q * m)
    out = torch.empty(nout, dtype=f.dtype, device=f.device)
    ws = ctypes.c_size_t(0)
    L = _native.lib()
    check(L.dc_workspace_size_pq(m, p, q, nout, dt, ctypes.byref(ws)), "dc_workspace_size_pq")
    work = _work(ws.value, f.device)
    check(L.dc_conv_complex_1d_pq(_vp(f), _vp(g), _vp(out), m, p, q, nout, dt, _vp(work), ws.value, _stream(f)),
          "dc_conv_complex_1d_pq")
    return out


def conv_complex_1d_full(f, g):
    """All 2m - 1 outputs of the linear convolution of two length-m inputs
    (general padding with p = 1, q = 2)."""
    return conv_complex_1d_pq(f, g, f.shape[0], 1, 2)


def conv_hermitian_1d(f, g, out=None):
    """Centered Hermitian 2/3-rule convolution (dc_conv_hermitian_1d)."""
    return _run_1d("dc_conv_hermitian_1d", KIND_HERMITIAN, [f, g], 1, None if out is None else [out])


def conv_ternary_hermitian_1d(f, g, e, out=None):
    """Centered Hermitian ternary convolution (dc_conv_ternary_hermitian_1d)."""
    return _run_1d("dc_conv_ternary_hermitian_1d", KIND_TERNARY, [f, g, e], 1,
                   None if out is None else [out])


def conv_complex_1d_adjoint(w, f, g):
    """(df, dg) of L = Re <w, conv_complex_1d(f, g)> (dc_conv_complex_1d_adjoint)."""
    return _run_1d("dc_conv_complex_1d_adjoint", KIND_COMPLEX_ADJOINT, [w, f, g], 2, None)


def conv_hermitian_1d_adjoint(w, f, g):
    """(df, dg) of L = Re <w, conv_hermitian_1d(f, g)> (dc_conv_hermitian_1d_adjoint)."""
    return _run_1d("dc_conv_hermitian_1d_adjoint", KIND_HERMITIAN_ADJOINT, [w, f, g], 2, None)


def _dims(t, hermitian):
    """Unpadded sizes of a multi-D array (centered Hermitian axes hold 2m-1)."""
    shape = list(t.shape)
    if not hermitian:
        return shape
    for n in shape[:-1]:
        if n % 2 != 1:
            raise ValueError("centered Hermitian axes hold 2m-1 entries")
    return [(n + 1) // 2 for n in shape[:-1]] + [shape[-1]]


def _run_md(name, kind, ins, nout, hermitian, slabs_per_chunk=None):
    dt = _inputs(*ins)
    if ins[0].dim() not in (2, 3):
        raise ValueError(f"{name}: expected 2D or 3D tensors")
    dims = _dims(ins[0], hermitian)
    outs = [torch.empty_like(ins[0]) for _ in range(nout)]
    if slabs_per_chunk is not None and len(dims) == 3:
        ws = workspace_size_slabs(kind, dims, dt, slabs_per_chunk)
    else:
        ws = workspace_size(kind, dims, dt)
    work = _work(ws, ins[0].device)
    fn = getattr(_native.lib(), name)
    args = [_vp(t) for t in ins] + [_vp(t) for t in outs] + list(dims)
    check(fn(*args, dt, _vp(work), ws, _stream(ins[0])), name)
    return outs[0] if nout == 1 else tuple(outs)


def _run_dot2(name, kind, ins, hermitian, slabs_per_chunk=None):
    dt = _inputs(*ins)
    if ins[0].dim() not in (1, 2, 3):
        raise ValueError(f"{name}: expected 1D, 2D or 3D tensors")
    dims = [ins[0].shape[0]] if ins[0].dim() == 1 else _dims(ins[0], hermitian)
    out = torch.empty_like(ins[0])
    if slabs_per_chunk is not None and len(dims) == 3:
        ws = workspace_size_slabs(kind, dims, dt, slabs_per_chunk)
    else:
        ws = workspace_size(kind, dims, dt)
    work = _work(ws, ins[0].device)
    d = (ctypes.c_int64 * len(dims))(*[int(x) for x in dims])
    fn = getattr(_native.lib(), name)
    check(fn(len(dims), d, *[_vp(t) for t in ins], _vp(out), dt, _vp(work), ws, _stream(ins[0])), name)
    return out


def conv_complex_dot2(f1, g1, f2, g2, slabs_per_chunk=None):
    """f1 * g1 + f2 * g2 for 1D/2D/3D complex convolutions with one forward
    transform per residue for both pairs (dc_conv_complex_dot2)."""
    return _run_dot2("dc_conv_complex_dot2", KIND_COMPLEX_DOT2, [f1, g1, f2, g2], False, slabs_per_chunk)


def conv_hermitian_dot2(f1, g1, f2, g2, slabs_per_chunk=None):
    """f1 * g1 + f2 * g2 for 1D/2D/3D centered Hermitian convolutions
    (dc_conv_hermitian_dot2); e.g. the 2D Euler advective term."""
    return _run_dot2("dc_conv_hermitian_dot2", KIND_HERMITIAN_DOT2, [f1, g1, f2, g2], True, slabs_per_chunk)


# slabs_per_chunk (3D only): a workspace sized for chunks of at most that
# many x-slabs (dc_workspace_size_slabs) instead of the default.

def conv_complex_nd(f, g, slabs_per_chunk=None):
    """2D/3D complex convolution (dc_conv_complex_2d / _3d)."""
    return _run_md(f"dc_conv_complex_{f.dim()}d", KIND_COMPLEX, [f, g], 1, False, slabs_per_chunk)


def conv_hermitian_nd(f, g, slabs_per_chunk=None):
    """2D/3D centered Hermitian convolution (dc_conv_hermitian_2d / _3d)."""
    return _run_md(f"dc_conv_hermitian_{f.dim()}d", KIND_HERMITIAN, [f, g], 1, True, slabs_per_chunk)


def conv_ternary_hermitian_nd(f, g, e, slabs_per_chunk=None):
    """2D/3D centered Hermitian ternary convolution (dc_conv_ternary_hermitian_2d / _3d)."""
    return _run_md(f"dc_conv_ternary_hermitian_{f.dim()}d", KIND_TERNARY, [f, g, e], 1, True, slabs_per_chunk)


def conv_complex_nd_adjoint(w, f, g, slabs_per_chunk=None):
    """(df, dg) for the 2D/3D complex convolution."""
    return _run_md(f"dc_conv_complex_{f.dim()}d_adjoint", KIND_COMPLEX_ADJOINT, [w, f, g], 2, False,
                   slabs_per_chunk)


def conv_hermitian_nd_adjoint(w, f, g, slabs_per_chunk=None):
    """(df, dg) for the 2D/3D centered Hermitian convolution."""
    return _run_md(f"dc_conv_hermitian_{f.dim()}d_adjoint", KIND_HERMITIAN_ADJOINT, [w, f, g], 2, True,
                   slabs_per_chunk)


def partition_lpt(sizes, nranks):
    """Owner rank of every instance and the per-rank summed costs
    (dc_partition_lpt: longest processing time first, cost m log2 m)."""
    n = len(sizes)
    m = (ctypes.c_int64 * max(n, 1))(*[int(x) for x in sizes])
    owner = (ctypes.c_int32 * max(n, 1))()
    load = (ctypes.c_double * int(nranks))()
    check(_native.lib().dc_partition_lpt(m, n, int(nranks), owner, load), "dc_partition_lpt")
    return [int(owner[i]) for i in range(n)], [float(load[r]) for r in range(int(nranks))]


def shard(sizes, rank, world):
    """Instance ids (in instance order) that rank `rank` of `world` convolves
    when one batch is split across processes by partition_lpt."""
    owner, _ = partition_lpt(sizes, world)
    return [i for i, o in enumerate(owner) if o == rank]


class BatchedPlan:
    """Plan for packed 1D complex convolutions of uneven sizes
    (dc_batched_plan_create / dc_conv_complex_1d_batched)."""

    def __init__(self, sizes, dtype=torch.complex64, flags=0):
        self.sizes = [int(x) for x in sizes]
        self.dtype = dtype
        self.code = C64 if dtype == torch.complex64 else C128
        arr = (ctypes.c_int64 * len(self.sizes))(*self.sizes)
        h = ctypes.c_void_p(0)
        check(_native.lib().dc_batched_plan_create(arr, len(self.sizes), self.code, flags, ctypes.byref(h)),
              "dc_batched_plan_create")
        self.handle = h
        ws = ctypes.c_size_t(0)
        check(_native.lib().dc_batched_plan_workspace_size(h, ctypes.byref(ws)), "workspace")
        self.workspace_bytes = int(ws.value)
        n = ctypes.c_int32(0)
        check(_native.lib().dc_batched_plan_launches(h, ctypes.byref(n)), "launches")
        self.launches = int(n.value)
        self.total = sum(self.sizes)
        self._work = None

    def describe(self):
        """Per distinct size: (m, level, instances per block, L1, L2, tile width)."""
        out = []
        i = 0
        while True:
            m, vals = ctypes.c_int64(0), [ctypes.c_int32(0) for _ in range(5)]
            st = _native.lib().dc_batched_plan_describe(self.handle, i, ctypes.byref(m),
                                                        *[ctypes.byref(v) for v in vals])
            if st != 0:
                break
            out.append((m.value,) + tuple(v.value for v in vals))
            i += 1
        return out

    def schedule(self):
        """(batch_target, l1_mode) of the fixed-shape engine's task queue, or
        None for plans on the runtime-shaped engine."""
        t, mo = ctypes.c_int32(0), ctypes.c_int32(0)
        if _native.lib().dc_batched_plan_schedule(self.handle, ctypes.byref(t), ctypes.byref(mo)) != 0:
            return None
        return t.value, mo.value

    def set_schedule(self, batch_target, l1_mode):
        """Rebuilds the task queue in the given order (dc_batched_plan_set_schedule)."""
        check(_native.lib().dc_batched_plan_set_schedule(self.handle, int(batch_target), int(l1_mode)),
              "dc_batched_plan_set_schedule")
        ws = ctypes.c_size_t(0)
        check(_native.lib().dc_batched_plan_workspace_size(self.handle, ctypes.byref(ws)), "workspace")
        self.workspace_bytes = int(ws.value)
        self._work = None

    def task_units(self):
        """Tiles or row groups per pass task (dc_batched_plan_task_units), or
        None for plans on the runtime-shaped engine."""
        u = ctypes.c_int32(0)
        if _native.lib().dc_batched_plan_task_units(self.handle, ctypes.byref(u)) != 0:
            return None
        return u.value

    def set_task_units(self, units):
        """Rebuilds the task queue with this many tiles or row groups per pass
        task (dc_batched_plan_set_task_units)."""
        check(_native.lib().dc_batched_plan_set_task_units(self.handle, int(units)),
              "dc_batched_plan_set_task_units")
        ws = ctypes.c_size_t(0)
        check(_native.lib().dc_batched_plan_workspace_size(self.handle, ctypes.byref(ws)), "workspace")
        self.workspace_bytes = int(ws.value)
        self._work = None

    def variants(self):
        """Bit mask of the size codes whose two-level split runs variant 1
        (dc_batched_plan_variants), or None for plans off the fixed engine."""
        v = ctypes.c_uint32(0)
        if _native.lib().dc_batched_plan_variants(self.handle, ctypes.byref(v)) != 0:
            return None
        return v.value

    def set_variants(self, mask):
        """Rebuilds the task queue with the given split variants
        (dc_batched_plan_set_variants)."""
        check(_native.lib().dc_batched_plan_set_variants(self.handle, int(mask) & 0xFFFFFFFF),
              "dc_batched_plan_set_variants")
        ws = ctypes.c_size_t(0)
        check(_native.lib().dc_batched_plan_workspace_size(self.handle, ctypes.byref(ws)), "workspace")
        self.workspace_bytes = int(ws.value)
        self._work = None

    def workspace(self, device):
        device = torch.device(device)
        if device.type == "cuda" and device.index is None:
            device = torch.device("cuda", torch.cuda.current_device())
        if self._work is None or self._work.device != device or self._work.numel() < self.workspace_bytes:
            self._work = _work(self.workspace_bytes, device)
        return self._work

    def __call__(self, f, g, out=None, work=None):
        _inputs(f, g)
        if f.dim() != 1 or f.shape[0] != self.total or f.dtype != self.dtype:
            raise ValueError("packed inputs must be 1D of the plan's total length and dtype")
        out = torch.empty_like(f) if out is None else out
        work = self.workspace(f.device) if work is None else work
        check(_native.lib().dc_conv_complex_1d_batched(self.handle, _vp(f), _vp(g), _vp(out), _vp(work),
                                                       work.numel(), _stream(f)),
              "dc_conv_complex_1d_batched")
        return out

    def host_workspace(self, nchunks, device):
        """Device workspace for run_from_host with this many chunks."""
        ws = ctypes.c_size_t(0)
        check(_native.lib().dc_batched_plan_host_workspace_size(self.handle, int(nchunks), ctypes.byref(ws)),
              "dc_batched_plan_host_workspace_size")
        return _work(ws.value, device)

    def run_from_host(self, hf, hg, hh, df, dg, dh, work, nchunks):
        """Host-to-host pipelined execution (dc_conv_complex_1d_batched_host):
        hf, hg, hh are CPU tensors (pinned), df, dg, dh CUDA tensors of the same
        packed layout; runs on the current stream."""
        for t in (hf, hg, hh):
            if t.is_cuda or t.dtype != self.dtype or t.numel() != self.total or not t.is_contiguous():
                raise ValueError("host arrays must be contiguous CPU tensors of the plan's size and dtype")
        for t in (df, dg, dh):
            if not t.is_cuda or t.dtype != self.dtype or t.numel() != self.total or not t.is_contiguous():
                raise ValueError("device arrays must be contiguous CUDA tensors of the plan's size and dtype")
        check(_native.lib().dc_conv_complex_1d_batched_host(
            self.handle, _vp(hf), _vp(hg), _vp(hh), _vp(df), _vp(dg), _vp(dh), _vp(work), work.numel(),
            int(nchunks), _stream(df)), "dc_conv_complex_1d_batched_host")
        return hh

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                _native.lib().dc_batched_plan_destroy(h)
            except Exception:
                pass
            self.handle = None

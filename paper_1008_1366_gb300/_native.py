"""ctypes loader for libdealias.so and the C signatures of include/dealias.h.

There is no fallback: if the library is missing or fails to load, importing
this module raises, naming the build step that produces it.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdealias.so")

_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_sz = ctypes.c_size_t

# name -> argument types (all return dc_status = int32 unless listed in _RET)
SIGNATURES = {
    "dc_status_string": [_i32],
    "dc_last_cuda_error": [],
    "dc_workspace_size": [_i32, _i32, ctypes.POINTER(_i64), _i32, ctypes.POINTER(_sz)],
    "dc_prepare": [_i32, _i32, ctypes.POINTER(_i64), _i32],
    "dc_workspace_size_slabs": [_i32, _i32, ctypes.POINTER(_i64), _i32, _i64, ctypes.POINTER(_sz)],
    "dc_chunking": [_i32, _i32, ctypes.POINTER(_i64), _i32, _sz, ctypes.POINTER(_i64), ctypes.POINTER(_i64)],
    "dc_read_status": [_vp, _vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32)],
    "dc_conv_complex_1d": [_vp, _vp, _vp, _i64, _i32, _vp, _sz, _vp],
    "dc_conv_hermitian_1d": [_vp, _vp, _vp, _i64, _i32, _vp, _sz, _vp],
    "dc_conv_ternary_hermitian_1d": [_vp, _vp, _vp, _vp, _i64, _i32, _vp, _sz, _vp],
    "dc_conv_complex_1d_adjoint": [_vp, _vp, _vp, _vp, _vp, _i64, _i32, _vp, _sz, _vp],
    "dc_conv_hermitian_1d_adjoint": [_vp, _vp, _vp, _vp, _vp, _i64, _i32, _vp, _sz, _vp],
    "dc_conv_complex_1d_noalloc": [_vp, _vp, _vp, _i64, _i32, _vp],
    "dc_conv_complex_dot2": [_i32, ctypes.POINTER(_i64)] + [_vp] * 5 + [_i32, _vp, _sz, _vp],
    "dc_conv_hermitian_dot2": [_i32, ctypes.POINTER(_i64)] + [_vp] * 5 + [_i32, _vp, _sz, _vp],
    "dc_conv_ternary_hermitian_2d": [_vp, _vp, _vp, _vp, _i64, _i64, _i32, _vp, _sz, _vp],
    "dc_conv_ternary_hermitian_3d": [_vp, _vp, _vp, _vp, _i64, _i64, _i64, _i32, _vp, _sz, _vp],
    "dc_workspace_size_pq": [_i64, _i32, _i32, _i64, _i32, ctypes.POINTER(_sz)],
    "dc_conv_complex_1d_pq": [_vp, _vp, _vp, _i64, _i32, _i32, _i64, _i32, _vp, _sz, _vp],
    "dc_conv_complex_2d": [_vp, _vp, _vp, _i64, _i64, _i32, _vp, _sz, _vp],
    "dc_conv_complex_3d": [_vp, _vp, _vp, _i64, _i64, _i64, _i32, _vp, _sz, _vp],
    "dc_conv_hermitian_2d": [_vp, _vp, _vp, _i64, _i64, _i32, _vp, _sz, _vp],
    "dc_conv_hermitian_3d": [_vp, _vp, _vp, _i64, _i64, _i64, _i32, _vp, _sz, _vp],
    "dc_conv_complex_2d_adjoint": [_vp, _vp, _vp, _vp, _vp, _i64, _i64, _i32, _vp, _sz, _vp],
    "dc_conv_complex_3d_adjoint": [_vp, _vp, _vp, _vp, _vp, _i64, _i64, _i64, _i32, _vp, _sz, _vp],
    "dc_conv_hermitian_2d_adjoint": [_vp, _vp, _vp, _vp, _vp, _i64, _i64, _i32, _vp, _sz, _vp],
    "dc_conv_hermitian_3d_adjoint": [_vp, _vp, _vp, _vp, _vp, _i64, _i64, _i64, _i32, _vp, _sz, _vp],
    "dc_batched_plan_create": [ctypes.POINTER(_i64), _i32, _i32, _i32, ctypes.POINTER(_vp)],
    "dc_batched_plan_workspace_size": [_vp, ctypes.POINTER(_sz)],
    "dc_batched_plan_launches": [_vp, ctypes.POINTER(_i32)],
    "dc_batched_plan_describe": [_vp, _i32, ctypes.POINTER(_i64)] + [ctypes.POINTER(_i32)] * 5,
    "dc_batched_plan_schedule": [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32)],
    "dc_batched_plan_set_schedule": [_vp, _i32, _i32],
    "dc_batched_plan_task_units": [_vp, ctypes.POINTER(_i32)],
    "dc_batched_plan_set_task_units": [_vp, _i32],
    "dc_batched_plan_variants": [_vp, ctypes.POINTER(ctypes.c_uint32)],
    "dc_batched_plan_set_variants": [_vp, ctypes.c_uint32],
    "dc_selftest_wait_timeout": [_vp, _sz, _i64, _vp],
    "dc_read_trace": [_vp, _vp, ctypes.POINTER(ctypes.c_uint64)],
    "dc_batched_plan_host_workspace_size": [_vp, _i32, ctypes.POINTER(_sz)],
    "dc_conv_complex_1d_batched_host": [_vp] + [_vp] * 7 + [_sz, _i32, _vp],
    "dc_conv_complex_1d_batched": [_vp, _vp, _vp, _vp, _vp, _sz, _vp],
    "dc_batched_plan_destroy": [_vp],
    "dc_partition_lpt": [ctypes.POINTER(_i64), _i32, _i32, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_double)],
}
_RET = {"dc_status_string": ctypes.c_char_p}


def load(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
            "(or python paper_1008_1366_gb300/build.py); there is no non-CUDA fallback")
    lib = ctypes.CDLL(path)
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = _RET.get(name, _i32)
    return lib


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = load()
    return _LIB

"""Builds the CUDA shared library (libdealias.so) in-tree for sm_103a.

Each .cu file is compiled by nvcc in parallel into _build/, then linked with
``nvcc -shared``.  Objects newer than every source and header are reused.
"""

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdealias.so")

SOURCES = ["capi.cu", "plan.cu", "twiddle.cu", "conv1d.cu", "batched.cu", "axis.cu", "multid.cu", "noalloc.cu",
           "partition.cu", "pq.cu"]
# the fixed-shape engine per precision: the outer-axis kernels, the batched
# planner, and the batched kernel of each convolution kind (MODE_* 0..5) in
# a translation unit of its own, so that the kinds compile in parallel
_PREC = (("f", "f32", "float2"), ("d", "f64", "double2"))
FIXED = ([("fixed_axis.cu", f"fixed_axis_{tag}.o", [f"-DDC_FX_P={ns}", f"-DDC_FX_C={c}"]) for tag, ns, c in _PREC]
         + [("fixed_batched.cu", f"fixed_batched_{tag}.o", [f"-DDC_FX_P={ns}", f"-DDC_FX_C={c}"])
            for tag, ns, c in _PREC]
         + [("fixed_batched.cu", f"fixed_batched_m{k}_{tag}.o", [f"-DDC_FX_P={ns}", f"-DDC_FX_C={c}",
                                                                 f"-DDC_FX_MODE={k}"])
            for k in range(6) for tag, ns, c in _PREC])
# the fused 1D kernel, one translation unit per (kind, precision)
INSTANCES = [(k, tag, c) for k in range(8) for tag, c in (("f", "float2"), ("d", "double2"))]


def _units():
    units = [(n, n.replace(".cu", ".o"), []) for n in SOURCES]
    for k, tag, c in INSTANCES:
        units.append(("conv1d_inst.cu", f"conv1d_k{k}_{tag}.o",
                      [f"-DDC_INST_KIND={k}", f"-DDC_INST_C={c}", f"-DDC_INST_TAG={tag}"]))
    for src, obj, defs in FIXED:
        units.append((src, obj, defs))
    return units


ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--use_fast_math=false"]


def _nvcc():
    path = shutil.which("nvcc")
    if path:
        return path
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdealias.so")


def _headers():
    hs = []
    for d in (CSRC, INCLUDE):
        for n in os.listdir(d):
            if n.endswith((".h", ".cuh")):
                hs.append(os.path.join(d, n))
    return hs


def _deps(obj, src, headers):
    """The sources and in-tree headers an object was compiled from: the
    dependency file nvcc wrote beside it (-MD), else every header."""
    dfile = obj + ".d"
    if not os.path.exists(dfile):
        return [src] + headers
    text = open(dfile).read().replace("\\\n", " ")
    parts = text.split(":", 1)[1].split() if ":" in text else []
    root = os.path.dirname(HERE)
    deps = [os.path.abspath(p) for p in parts if os.path.abspath(p).startswith(root)]
    return deps or [src] + headers


def _stale(obj, src, headers):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = _deps(obj, src, headers)
    return any(not os.path.exists(p) or os.path.getmtime(p) > t for p in deps)


def build(verbose=False, jobs=None, extra_flags=()):
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    headers = _headers()
    flags = [f for f in FLAGS if not f.startswith("--use_fast_math")] + list(extra_flags)

    def compile_one(unit):
        name, objname, defs = unit
        src = os.path.join(CSRC, name)
        obj = os.path.join(BUILD, objname)
        if not _stale(obj, src, headers):
            return obj, ""
        cmd = [nvcc] + ARCH + flags + defs + ["-I", INCLUDE, "-MD", "-MF", obj + ".d", "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {objname}:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return obj, r.stdout + r.stderr

    units = _units()
    jobs = jobs or min(len(units), os.cpu_count() or 4)
    # longest units first: the fixed-shape engine, then the fused kernels
    units.sort(key=lambda u: 0 if "_m" in u[1] and u[0] == "fixed_batched.cu" else (1 if u[0] == "conv1d_inst.cu" else 2))
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(compile_one, units))
    objs = [o for o, _ in results]
    if verbose:
        for _, log in results:
            if log:
                sys.stderr.write(log)
    if not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        cmd = [nvcc] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))

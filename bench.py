"""Benchmark: batched FP32 implicitly dealiased 1D complex convolutions.

Workload (the one the headline metric is quoted on): 4096 independent 1D
complex binary convolutions, m drawn uniformly from the 31 sizes
{2^k, 3*2^k, 5*2^k} in [64, 65536] (seed 1012), entries uniform[-1, 1],
complex64, executed as ONE persistent kernel launch replayed from a CUDA
graph.  A step is one such call over the whole batch.  Reported beside it:
the plain FP64 path (one launch per instance), parity against the FP64
oracle on sampled instances, the HBM roofline of the kernel and the CPU
oracle on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) the N ranks convolve one batch of 4096 N instances,
split by the longest-processing-time partition of the library
(dc_partition_lpt, cost m log2 m): each rank plans and runs its own share,
with no collective on the data path (weak scaling: about 4096 instances per
rank); rank 0 prints the aggregate over the slowest rank's time.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_INST = 4096
SEED = 1012
WORKLOAD = ("batched 1D complex binary implicitly dealiased convolution: 4096 instances, "
            "m uniform over {2^k,3*2^k,5*2^k} in [64,65536], uniform[-1,1] entries, complex64, "
            "one persistent launch in a CUDA graph")
METRIC = "dealiased convs/s (FP32 batched, one persistent launch)"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--suite", action="store_true",
                   help="measure every configuration of the scope but the batched one, one JSON line each")
    p.add_argument("--suite-only", default=None,
                   help="with --suite: only the configurations whose name contains this text, "
                        "'_' standing for a space (e.g. 3D_Hermitian; for profiling one of them)")
    p.add_argument("--no-suite", action="store_true",
                   help="leave the other configurations out of the headline line")
    p.add_argument("--variants", default=None,
                   help="with --per-size: split-variant mask of the two-level sizes (e.g. 0xffffffff)")
    p.add_argument("--per-size", default=None,
                   help="comma-separated sizes (or 'all' for the 31 of the workload): time one-size "
                        "batches of about 16 M elements each on the fixed-shape engine, one JSON line "
                        "per size (ps per element; for profiling one size alone)")
    p.add_argument("--instances", type=int, default=N_INST,
                   help="batch size (default 4096; smaller batches are for profiling only)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def global_sizes(world, n=N_INST):
    """Sizes of the whole batch: n instances per rank, one seeded draw."""
    from paper_1008_1366_gb300 import synthetic
    return synthetic.batched_sizes(n * world, SEED)


def workload(ids, sizes):
    """This share's sizes and packed inputs (each instance from its own
    seeded stream, so a share is generated alone)."""
    from paper_1008_1366_gb300 import synthetic
    ms = np.asarray([int(sizes[i]) for i in ids], dtype=np.int64)
    f, g, off = synthetic.instance_inputs(sizes, ids, SEED + 7)
    return ms, f, g, off


def oracle_convs(ms, f, g, off, budget_s, start=0):
    """Times the FP64 oracle over instances start, start+1, ... (cyclic) until
    budget_s seconds of CPU work; returns (convs, seconds, sample text)."""
    import oracle
    n = len(ms)
    t0 = time.perf_counter()
    done = 0
    elems = 0
    while True:
        i = (start + done) % n
        a, b = off[i], off[i + 1]
        oracle.padded_complex(f[a:b], g[a:b])
        done += 1
        elems += int(b - a)
        if time.perf_counter() - t0 >= budget_s or done >= 4 * n:
            break
    dt = time.perf_counter() - t0
    return done, dt, (f"{done} instances of the workload in order (sum m = {elems}), "
                      f"explicitly padded FFT convolution ({oracle.conv.FFT_LIBRARY}), 1 process")


def _oracle_worker(args):
    """One process of the all-cores CPU baseline: generates instances
    ids[start], ids[start + stride], ... of the batch (outside its clock),
    then convolves them with the FP64 oracle, in order and cyclically, for
    budget_s seconds; returns (convs, elements, seconds)."""
    sizes, ids, start, stride, budget_s = args
    import oracle
    from paper_1008_1366_gb300 import synthetic
    mine = ids[start::stride]
    if not mine:
        return 0, 0, 0.0
    f, g, off = synthetic.instance_inputs(sizes, mine, SEED + 7)
    t0 = time.perf_counter()
    done = elems = 0
    while True:
        j = done % len(mine)
        a, b = off[j], off[j + 1]
        oracle.padded_complex(f[a:b], g[a:b])
        done += 1
        elems += int(b - a)
        if time.perf_counter() - t0 >= budget_s:
            break
    return done, elems, time.perf_counter() - t0


def oracle_convs_all_cores(sizes, ids, budget_s):
    """The oracle on every host core this process may use: a spawned pool of
    one process per core, each taking every cores-th instance of the share.
    Returns (convs/s over the slowest process's time, cores, sample text)."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    jobs = [(sizes, list(ids), k, cores, budget_s) for k in range(cores)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, jobs)
    done = sum(r[0] for r in res)
    elems = sum(r[1] for r in res)
    dt = max(r[2] for r in res)
    return done / dt, cores, (f"{done} instance convolutions of the workload (sum m = {elems}) on {cores} "
                              f"processes (spawned pool, instances strided over the processes, about "
                              f"{budget_s:.0f} s each), explicitly padded FFT convolution")


class Clocks:
    """Samples nvidia-smi during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        if self.proc:
            time.sleep(1.0)   # nvidia-smi's first sample lands about a second after start
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# the translation unit of fx_kernel: its source and every header it includes
FX_KERNEL_SOURCES = ["paper_1008_1366_gb300/csrc/fixed_batched.cu", "paper_1008_1366_gb300/csrc/fixed.cuh",
                     "paper_1008_1366_gb300/csrc/fixed.h", "paper_1008_1366_gb300/csrc/fft2.cuh",
                     "paper_1008_1366_gb300/csrc/fft.cuh", "paper_1008_1366_gb300/csrc/common.cuh",
                     "paper_1008_1366_gb300/csrc/launch.h", "include/dealias.h"]


def kernel_source_hash():
    h = hashlib.sha256()
    for n in FX_KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, n), "rb").read())
    return h.hexdigest()[:16]


def committed_traffic(total_bytes_alg):
    """DRAM traffic per launch from the committed ncu summary, if it was taken
    on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    if rec.get("source_hash") != kernel_source_hash():
        return None
    if rec.get("alg_bytes_per_launch") != total_bytes_alg:   # another workload
        return None
    return rec.get("traffic_bytes_per_launch")


def measured_peak_hbm():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def run_reference(args, rank, world):
    if rank != 0:
        return
    sizes = global_sizes(1)
    ms, f, g, off = workload(list(range(len(sizes))), sizes)
    times, convs = [], []
    cores = 1
    for s in range(args.warmup + args.steps):
        n, dt, sample = oracle_convs(ms, f, g, off, budget_s=3.0, start=s * 64)
        if s >= args.warmup:
            times.append(dt)
            convs.append(n)
    value = sum(convs) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "convs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD + " (bounded sample per step)"},
        "cpu_baseline": {"value": value, "unit": "convs/s", "cores": cores, "kind": "oracle",
                         "sample": "each step: about 3 s of the workload's instances in order (the FP64 "
                                   "oracle, 1 process); last step: " + sample},
        "e2e": {"value": value, "unit": "convs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _time_call(fn, reps, warm=2):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts), ts


def one_sided_sigma(ts):
    """Mean T and the one-sided deviations sigma_L, sigma_H (Sec. 2.1 timing
    statistic, read with the square root over the whole quotient)."""
    T = statistics.mean(ts)
    n = len(ts)
    d = max(n / 2 - 1, 1)
    lo = sum((t - T) ** 2 for t in ts if t < T)
    hi = sum((t - T) ** 2 for t in ts if t > T)
    return T, (lo / d) ** 0.5, (hi / d) ** 0.5


def _pointwise_ratio(got, ref, N, u, scale):
    """Largest output error over the pointwise bar of the parity tests:
    8 u log2(N) (2 S + 2 ||ref||) + 4 u S, S the inputs' norm product."""
    got = np.asarray(got, dtype=np.complex128).ravel()
    ref = np.asarray(ref, dtype=np.complex128).ravel()
    bar = 8.0 * u * np.log2(max(N, 2)) * (2.0 * scale + 2.0 * np.linalg.norm(ref)) + 4.0 * u * scale
    return float(np.max(np.abs(got - ref)) / bar)


def run_suite(args, only=None, peak=None):
    """Every configuration of the scope but the batched one: time (CUDA
    events, median of reps, mean with the one-sided sigma_L / sigma_H),
    convolutions/s, algorithmic GB/s and fraction of the measured HBM peak,
    and parity against the FP64 oracle over every output (relative L2 and
    the pointwise bar).  Returns one record per configuration."""
    import torch
    import oracle
    import paper_1008_1366_gb300 as dcl
    from paper_1008_1366_gb300 import synthetic
    from oracle.adjoint import symmetrize_upstream
    if peak is None:
        peak, _ = measured_peak_hbm()
    dev = torch.device("cuda", torch.cuda.current_device())
    out = []

    def want(name):
        # `only` matches a name's text, '_' standing for a space
        return only is None or only.replace("_", " ") in name

    def emit(name, ms, ts, nbytes, err, tol, pw=None, extra=None):
        T, sl, sh = one_sided_sigma(ts)
        rec = {"config": name, "ms_median": ms, "ms_mean": T, "sigma_L": sl, "sigma_H": sh, "runs": len(ts),
               "convs_per_s": 1e3 / ms, "alg_bytes": nbytes, "gbs": nbytes / ms / 1e6,
               "hbm_frac_of_measured": nbytes / ms / 1e6 / peak, "rel_l2": err, "tol": tol,
               "pointwise_over_bar": pw, "parity_ok": (err is not None and err <= tol and (pw is None or pw <= 1.0))}
        if extra:
            rec.update(extra)
        out.append(rec)

    def rel(a, b):
        a = np.asarray(a, dtype=np.complex128).ravel()
        b = np.asarray(b, dtype=np.complex128).ravel()
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    def nrm(*arrs):
        return float(np.prod([np.linalg.norm(np.asarray(a).ravel()) for a in arrs]))

    def hnrm(*arrs):
        return nrm(*[oracle.hermitian_extend(oracle.project_hermitian(a)) for a in arrs])

    U = {torch.complex64: 2.0 ** -24, torch.complex128: 2.0 ** -53}
    reps = max(20, min(args.steps, 200))
    if want("1D complex"):
        f = synthetic.uniform_complex(1024, 1009)
        g = synthetic.uniform_complex(1024, 1010)
        tf, tg = (torch.tensor(x, dtype=torch.complex128, device=dev) for x in (f, g))
        ms, ts = _time_call(lambda: dcl.conv_complex_1d(tf, tg), reps)
        h, ref = dcl.conv_complex_1d(tf, tg).cpu().numpy(), oracle.direct_complex(f, g)
        emit("1D complex m=1024 c128", ms, ts, 3 * 1024 * 16, rel(h, ref), 1e-12,
             _pointwise_ratio(h, ref, 2048, U[torch.complex128], nrm(f, g)))
    if want("1D Hermitian"):
        m = 1 << 16
        f = synthetic.hermitian_spectrum((m,), 1.0, 1010)
        g = synthetic.hermitian_spectrum((m,), 1.0, 1011)
        ref = oracle.padded_hermitian(f, g)
        for dt, tol in ((torch.complex128, 1e-12), (torch.complex64, 5e-7 * np.log2(3 * m))):
            tf, tg = (torch.tensor(x, dtype=dt, device=dev) for x in (f, g))
            ms, ts = _time_call(lambda: dcl.conv_hermitian_1d(tf, tg), reps)
            h = dcl.conv_hermitian_1d(tf, tg).cpu().numpy()
            emit(f"1D Hermitian m=2^16 {str(dt)[6:]}", ms, ts, 3 * m * tf.element_size(), rel(h, ref), tol,
                 _pointwise_ratio(h, ref, 3 * m, U[dt], hnrm(f, g)))
    if want("1D ternary"):
        m = 1 << 14
        fs = [synthetic.hermitian_spectrum((m,), 1.0, 1010 + s) for s in range(3)]
        ref = oracle.padded_ternary_hermitian(*fs)
        ext = [oracle.hermitian_extend(oracle.project_hermitian(a)) for a in fs]
        n2 = [np.linalg.norm(a) for a in ext]
        n1 = [np.abs(a).sum() for a in ext]
        S3 = n2[0] * n2[1] * n1[2] + n2[0] * n2[2] * n1[1] + n2[1] * n2[2] * n1[0]
        for dt, tol in ((torch.complex128, 1e-12), (torch.complex64, 5e-7 * np.log2(4 * m))):
            ts_ = [torch.tensor(x, dtype=dt, device=dev) for x in fs]
            ms, ts = _time_call(lambda: dcl.conv_ternary_hermitian_1d(*ts_), reps)
            h = dcl.conv_ternary_hermitian_1d(*ts_).cpu().numpy()
            emit(f"1D ternary Hermitian m=2^14 {str(dt)[6:]}", ms, ts, 4 * m * ts_[0].element_size(), rel(h, ref),
                 tol, _pointwise_ratio(h, ref, 4 * m, U[dt], S3))
    if want("2D Hermitian"):
        shape = synthetic.hermitian_shape((1024, 1024))
        f = synthetic.hermitian_spectrum(shape, 1.5, 1011)
        g = synthetic.hermitian_spectrum(shape, 1.5, 1012)
        tf, tg = (torch.tensor(x, dtype=torch.complex64, device=dev) for x in (f, g))
        ms, ts = _time_call(lambda: dcl.conv_hermitian_nd(tf, tg), reps)
        h, ref = dcl.conv_hermitian_nd(tf, tg).cpu().numpy(), oracle.padded_hermitian(f, g)
        N = 9 * 1024 * 1024
        emit("2D Hermitian 2047x1024 c64", ms, ts, 3 * f.size * 8, rel(h, ref), 5e-7 * np.log2(N),
             _pointwise_ratio(h, ref, N, U[torch.complex64], hnrm(f, g)))
    if want("2D complex"):
        f = synthetic.uniform_complex((2048, 2048), 1013)
        g = synthetic.uniform_complex((2048, 2048), 1014)
        tf, tg = (torch.tensor(x, dtype=torch.complex64, device=dev) for x in (f, g))
        ms, ts = _time_call(lambda: dcl.conv_complex_nd(tf, tg), reps)
        h, ref = dcl.conv_complex_nd(tf, tg).cpu().numpy(), oracle.padded_complex(f, g)
        N = 4 * 2048 * 2048
        emit("2D complex 2048x2048 c64", ms, ts, 3 * f.size * 8, rel(h, ref), 5e-7 * np.log2(N),
             _pointwise_ratio(h, ref, N, U[torch.complex64], nrm(f, g)))
    if want("2D ternary"):
        # next row f1: the 2D ternary Hermitian convolution at the shape of the
        # paper's Fig. 9 (mx = my = 4096), N = 4m per axis
        ms2 = (4096, 4096)
        shape = synthetic.hermitian_shape(ms2)
        fs = [synthetic.hermitian_spectrum(shape, 1.5, 1030 + s_) for s_ in range(3)]
        ts_ = [torch.tensor(x, dtype=torch.complex64, device=dev) for x in fs]
        ms, ts = _time_call(lambda: dcl.conv_ternary_hermitian_nd(*ts_), max(5, reps // 4))
        h = dcl.conv_ternary_hermitian_nd(*ts_).cpu().numpy()
        ref = oracle.padded_ternary_hermitian(*fs)
        ext = [oracle.hermitian_extend(oracle.project_hermitian(a)) for a in fs]
        n2 = [np.linalg.norm(a) for a in ext]
        n1 = [np.abs(a).sum() for a in ext]
        S3 = n2[0] * n2[1] * n1[2] + n2[0] * n2[2] * n1[1] + n2[1] * n2[2] * n1[0]
        N = 16 * 4096 * 4096
        emit("2D ternary Hermitian 8191x4096 c64", ms, ts, 4 * fs[0].size * 8, rel(h, ref), 5e-7 * np.log2(N),
             _pointwise_ratio(h, ref, N, U[torch.complex64], S3))
        del h, ref, ext, ts_
    if want("2D Euler"):
        # next row f2: the 2D Euler advective term as one dot product of two
        # pairs, beside the two separate convolutions it replaces
        shape = synthetic.hermitian_shape((1024, 1024))
        w = synthetic.hermitian_spectrum(shape, 1.5, 1040)
        kx = (np.arange(shape[0]) - 1023)[:, None] * np.ones((1, shape[1]))
        ky = np.ones((shape[0], 1)) * np.arange(shape[1])[None, :]
        k2 = kx ** 2 + ky ** 2
        inv = np.where(k2 > 0, 1.0 / np.where(k2 > 0, k2, 1.0), 0.0)
        fs = [1j * kx * w, 1j * ky * w]
        gs = [1j * ky * w * inv, -1j * kx * w * inv]
        tf = [torch.tensor(x, dtype=torch.complex64, device=dev) for x in fs]
        tg = [torch.tensor(x, dtype=torch.complex64, device=dev) for x in gs]
        ms, ts = _time_call(lambda: dcl.conv_hermitian_dot2(tf[0], tg[0], tf[1], tg[1]), reps)
        ms_sep, _ = _time_call(lambda: (dcl.conv_hermitian_nd(tf[0], tg[0]), dcl.conv_hermitian_nd(tf[1], tg[1])), reps)
        h = dcl.conv_hermitian_dot2(tf[0], tg[0], tf[1], tg[1]).cpu().numpy()
        ref = oracle.dot_hermitian(fs, gs)
        N = 9 * 1024 * 1024
        emit("2D Euler advective term (Hermitian dot product of two pairs) 2047x1024 c64", ms, ts,
             5 * w.size * 8, rel(h, ref), 5e-7 * np.log2(N),
             _pointwise_ratio(h, ref, N, U[torch.complex64], hnrm(fs[0], gs[0]) + hnrm(fs[1], gs[1])),
             {"ms_two_separate_convolutions": ms_sep})
    if want("1D complex full"):
        # next row f3: general padding, the full 2m - 1 outputs (p = 1, q = 2)
        m = 8192
        f = synthetic.uniform_complex(m, 1041)
        g = synthetic.uniform_complex(m, 1042)
        tf, tg = (torch.tensor(x, dtype=torch.complex64, device=dev) for x in (f, g))
        ms, ts = _time_call(lambda: dcl.conv_complex_1d_full(tf, tg), reps)
        h = dcl.conv_complex_1d_full(tf, tg).cpu().numpy()
        ref = oracle.padded_complex_pq(f, g, m, 2, 2 * m - 1)
        emit("1D complex full 2m-1 output (p/q = 1/2) m=8192 c64", ms, ts, (2 * m + 2 * m - 1) * 8, rel(h, ref),
             5e-7 * np.log2(2 * m), _pointwise_ratio(h, ref, 2 * m, U[torch.complex64], nrm(f, g)))
    if want("2D Hermitian odd"):
        # next row f4: odd m = 2c + 1 on both axes (405 = 5 x 3^4)
        ms2 = (405, 405)
        shape = synthetic.hermitian_shape(ms2)
        f = synthetic.hermitian_spectrum(shape, 1.5, 1043)
        g = synthetic.hermitian_spectrum(shape, 1.5, 1044)
        tf, tg = (torch.tensor(x, dtype=torch.complex64, device=dev) for x in (f, g))
        ms, ts = _time_call(lambda: dcl.conv_hermitian_nd(tf, tg), reps)
        h, ref = dcl.conv_hermitian_nd(tf, tg).cpu().numpy(), oracle.padded_hermitian(f, g)
        N = 9 * 405 * 405
        emit("2D Hermitian odd m 809x405 c64", ms, ts, 3 * f.size * 8, rel(h, ref), 5e-7 * np.log2(N),
             _pointwise_ratio(h, ref, N, U[torch.complex64], hnrm(f, g)))
    if want("3D Hermitian"):
        shape = synthetic.hermitian_shape((256, 256, 256))
        N = 27 * 256 ** 3
        f = synthetic.hermitian_spectrum(shape, 11 / 6, 1015)
        g = synthetic.hermitian_spectrum(shape, 11 / 6, 1016)
        w = synthetic.uniform_complex(shape, 1017)
        tf, tg, tw = (torch.tensor(x, dtype=torch.complex64, device=dev) for x in (f, g, w))
        ms, ts = _time_call(lambda: dcl.conv_hermitian_nd(tf, tg), max(5, reps // 4))
        h = dcl.conv_hermitian_nd(tf, tg).cpu().numpy()
        ref = oracle.padded_hermitian(f, g)
        emit("3D Hermitian 511x511x256 c64 forward", ms, ts, 3 * f.size * 8, rel(h, ref), 5e-7 * np.log2(N),
             _pointwise_ratio(h, ref, N, U[torch.complex64], hnrm(f, g)))
        del h, ref
        ms, ts = _time_call(lambda: dcl.conv_hermitian_nd_adjoint(tw, tf, tg), max(5, reps // 4))
        df, dg = (x.cpu().numpy() for x in dcl.conv_hermitian_nd_adjoint(tw, tf, tg))
        rdf, rdg = oracle.adjoint_hermitian(w, f, g)
        W = symmetrize_upstream(w)
        e = max(rel(df, rdf), rel(dg, rdg))
        pw = max(_pointwise_ratio(df, rdf, N, U[torch.complex64], hnrm(W, g)),
                 _pointwise_ratio(dg, rdg, N, U[torch.complex64], hnrm(W, f)))
        emit("3D Hermitian 511x511x256 c64 backward (df, dg)", ms, ts, 5 * f.size * 8, e, 5e-7 * np.log2(N), pw)
    return out


def per_size_rates(sizes, reps, warm, variants=None, elems=1 << 24):
    """One-size batches of about `elems` elements (FP32, default queue order,
    no autotuning): time per launch and ps per element, one record per size.
    Separates a size's own cost from the cost of mixing sizes in one launch."""
    import torch
    import paper_1008_1366_gb300 as dcl
    dev = torch.device("cuda", torch.cuda.current_device())
    out_recs = []
    for m in sizes:
        n = max(1, elems // m)
        f = torch.rand(n * m, dtype=torch.complex64, device=dev)
        g = torch.rand(n * m, dtype=torch.complex64, device=dev)
        plan = dcl.BatchedPlan([m] * n, dtype=torch.complex64)
        if variants:
            plan.set_variants(int(variants, 0))
        out = torch.empty_like(f)
        work = plan.workspace(dev)
        ms, ts = _time_call(lambda: plan(f, g, out=out, work=work), reps, warm=warm)
        d = plan.describe()[0]
        out_recs.append({"m": m, "instances": n, "ms_median": ms, "ps_per_element": ms * 1e9 / (n * m),
                         "level": d[1], "split": "%dx%d" % (d[3], d[4]) if d[1] == 2 else None})
        del f, g, out, work, plan
    return out_recs


def run_per_size(args):
    """`--per-size`: one JSON line per size (per_size_rates)."""
    from paper_1008_1366_gb300 import synthetic
    sizes = synthetic.SIZES_31 if args.per_size == "all" else [int(x) for x in args.per_size.split(",")]
    for rec in per_size_rates(sizes, max(3, args.steps), max(3, args.warmup), args.variants):
        print(json.dumps(rec), flush=True)


def cufft_padded_context(ms, tf, tg, stream, reps=5):
    """Context only (not the product path): the conventional explicitly
    zero-padded convolution of the same batch on cuFFT through torch.fft,
    instances grouped by size, N = 2m, with the gathers and scatters of the
    packed layout.  Returns ms per batch and the max |difference| to th."""
    import torch
    dev = tf.device
    off = np.concatenate([[0], np.cumsum(ms)])
    groups = {}
    for i, m in enumerate(ms):
        groups.setdefault(int(m), []).append(int(off[i]))
    idx = {m: (torch.tensor(starts, device=dev)[:, None] + torch.arange(m, device=dev)[None, :])
           for m, starts in groups.items()}
    out = torch.empty_like(tf)

    def run():
        for m, ix in idx.items():
            F = torch.fft.fft(tf[ix], n=2 * m)
            G = torch.fft.fft(tg[ix], n=2 * m)
            out[ix] = torch.fft.ifft(F * G)[:, :m]

    with torch.cuda.stream(stream):
        run()
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            run()
        e1.record(stream)
    stream.synchronize()
    return e0.elapsed_time(e1) / reps, out


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.suite:
        import torch
        torch.cuda.set_device(local)
        for rec in run_suite(args, only=args.suite_only):
            print(json.dumps(rec), flush=True)
        return
    if args.per_size:
        import torch
        torch.cuda.set_device(local)
        run_per_size(args)
        return

    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    import oracle
    import paper_1008_1366_gb300 as dcl

    # one batch of instances per rank, split across the ranks by cost (LPT)
    sizes = global_sizes(world, args.instances)
    owner, loads = dcl.partition_lpt(sizes, world)
    ids = [i for i, o in enumerate(owner) if o == rank]
    ms, f, g, off = workload(ids, sizes)
    n_inst = len(ms)
    total = int(off[-1])
    tf = torch.tensor(f, dtype=torch.complex64, device=dev)
    tg = torch.tensor(g, dtype=torch.complex64, device=dev)
    th = torch.empty_like(tf)
    plan = dcl.BatchedPlan(ms, dtype=torch.complex64, flags=dcl.api.PLAN_AUTOTUNE)
    work = plan.workspace(dev)
    stream = torch.cuda.Stream(device=dev)

    # parity on sampled instances (outside the timed region)
    with torch.cuda.stream(stream):
        plan(tf, tg, out=th, work=work)
    stream.synchronize()
    hh = th.cpu().numpy()
    rng = np.random.default_rng(5)
    pick = sorted(set(rng.integers(0, len(ms), 24).tolist()) | {int(np.argmax(ms)), int(np.argmin(ms))})
    worst = worst_ratio = worst_pw = 0.0
    refs = {}
    for i in pick:
        a, b = off[i], off[i + 1]
        ref = refs[i] = oracle.padded_complex(f[a:b], g[a:b])
        e = float(np.linalg.norm(hh[a:b] - ref) / np.linalg.norm(ref))
        tol = 5e-7 * np.log2(2 * ms[i])
        worst = max(worst, e)
        worst_ratio = max(worst_ratio, e / tol)
        worst_pw = max(worst_pw, _pointwise_ratio(hh[a:b], ref, 2 * ms[i], 2.0 ** -24,
                                                  float(np.linalg.norm(f[a:b]) * np.linalg.norm(g[a:b]))))

    # capture one step in a CUDA graph
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        plan(tf, tg, out=th, work=work)
        stream.synchronize()
        with torch.cuda.graph(graph, stream=stream):
            plan(tf, tg, out=th, work=work)
    stream.synchronize()

    def step():
        graph.replay()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    th.zero_()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            for k in range(args.steps):
                step()
                ev[k + 1].record(stream)
        stream.synchronize()
    torch.cuda.synchronize()
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    t_ms = ev[0].elapsed_time(ev[-1])
    if pg:
        t = torch.tensor([t_ms], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        t_ms = float(t.item())
        pg.barrier()
    # the graph replays' output is the eager launch's, bit for bit
    replay_ok = bool(np.array_equal(th.cpu().numpy(), hh))
    # where the kernel's blocks spent their cycles (last launch of the loop)
    trace = dcl.read_trace(work)
    busy = sum(trace["cycles"].values())
    # block-cycles of the launch: blocks x duration x SM clock (sampled)
    clk_mhz = clk.summary().get("sm_mhz") or 2070.0
    # (the FP32 fixed-shape kernel runs two blocks per SM)
    launch_cycles = 2 * torch.cuda.get_device_properties(dev).multi_processor_count * \
        statistics.mean(per) * 1e-3 * clk_mhz * 1e6
    trace = {"tasks": trace["tasks"], "cycle_share": {k: round(v / max(1, busy), 4) for k, v in trace["cycles"].items()},
             "tasks_that_waited": trace["waited"], "wait_cycles_over_task_cycles": round(trace["wait_cycles"] / max(1, busy), 5),
             "block_time_share": {"in_tasks": round(busy / launch_cycles, 4),
                                  "handover": round(trace["handover_cycles"] / launch_cycles, 4),
                                  "root_tables": round(trace["table_cycles"] / launch_cycles, 4)}}
    convs_total = len(sizes) * args.steps
    value = convs_total / (t_ms / 1e3)
    ms_step = t_ms / args.steps
    T_mean, sig_l, sig_h = one_sided_sigma(per)

    # end to end through the public API with pinned host buffers: the
    # host-to-host call (dc_conv_complex_1d_batched_host) copies chunks of
    # instances in, convolves and copies out on overlapping streams; every
    # step copies all inputs in and all results out.  The chunk count is the
    # best of a few, each timed on its own.
    hf = torch.tensor(f, dtype=torch.complex64).pin_memory()
    hg = torch.tensor(g, dtype=torch.complex64).pin_memory()
    hout = torch.empty_like(hf).pin_memory()
    e2e_steps = max(3, min(args.steps, 10))
    e2e_best = None
    for nchunks in (1, 8, 16, 32):
        hw = plan.host_workspace(nchunks, dev)
        if pg:
            pg.barrier()
        with torch.cuda.stream(stream):
            for k in range(2 + e2e_steps):
                if k == 2:
                    stream.synchronize()
                    t0 = time.perf_counter()
                plan.run_from_host(hf, hg, hout, tf, tg, th, hw, nchunks)
            stream.synchronize()
            e2e_s = time.perf_counter() - t0
        if pg:
            t = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            e2e_s = float(t.item())
        val = len(sizes) * e2e_steps / e2e_s
        if e2e_best is None or val > e2e_best[0]:
            e2e_best = (val, nchunks)
        del hw
    e2e_val, e2e_chunks = e2e_best
    e2e_ok = bool(np.array_equal(hout.numpy(), hh))

    # plain FP64 path: one launch per instance
    fp64 = None
    if not args.no_fp64 and rank == 0:
        plan64 = dcl.BatchedPlan(ms, dtype=torch.complex128, flags=dcl.api.PLAN_ONE_PER_LAUNCH)
        tf64 = torch.tensor(f, dtype=torch.complex128, device=dev)
        tg64 = torch.tensor(g, dtype=torch.complex128, device=dev)
        th64 = torch.empty_like(tf64)
        w64 = plan64.workspace(dev)
        with torch.cuda.stream(stream):
            plan64(tf64, tg64, out=th64, work=w64)
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan64(tf64, tg64, out=th64, work=w64)
            e1.record(stream)
        stream.synchronize()
        t64 = e0.elapsed_time(e1)
        h64 = th64.cpu().numpy()
        worst64 = max(float(np.linalg.norm(h64[off[i]:off[i + 1]] - refs[i]) / np.linalg.norm(refs[i])) for i in pick)
        fp64 = {"convs_per_s": n_inst / (t64 / 1e3), "ms_per_batch": t64, "launches": plan64.launches,
                "max_rel_l2_sampled": worst64, "tol": 1e-12}
        del w64, plan64
        # the same FP64 arithmetic batched in one launch (context for the
        # precision cost alone)
        planb = dcl.BatchedPlan(ms, dtype=torch.complex128)
        wb = planb.workspace(dev)
        with torch.cuda.stream(stream):
            for _ in range(3):
                planb(tf64, tg64, out=th64, work=wb)
            e0.record(stream)
            for _ in range(5):
                planb(tf64, tg64, out=th64, work=wb)
            e1.record(stream)
        stream.synchronize()
        tb = e0.elapsed_time(e1) / 5
        hb = th64.cpu().numpy()
        worstb = max(float(np.linalg.norm(hb[off[i]:off[i + 1]] - refs[i]) / np.linalg.norm(refs[i])) for i in pick)
        fp64["batched_one_launch"] = {"convs_per_s": n_inst / (tb / 1e3), "ms_per_batch": tb,
                                      "max_rel_l2_sampled": worstb}
        del tf64, tg64, th64, wb, planb

    # context: the explicitly zero-padded convolution on cuFFT (torch.fft)
    cufft = None
    if rank == 0:
        tc, hc = cufft_padded_context(ms, tf, tg, stream)
        cufft = {"ms_per_batch": tc, "convs_per_s": n_inst / (tc / 1e3),
                 "max_rel_l2_vs_implicit_sampled": max(
                     float(np.linalg.norm(hc[off[i]:off[i + 1]].cpu().numpy() - refs[i]) / np.linalg.norm(refs[i]))
                     for i in pick),
                 "what": "explicitly zero-padded FFT convolution (N = 2m) on cuFFT via torch.fft, instances "
                         "grouped by size, gathers and scatters of the packed layout included; context only"}
        del hc

    cpu = None
    if not args.no_cpu and rank == 0:
        n, dt, sample = oracle_convs(ms, f, g, off, budget_s=10.0)
        cpu = {"value": n / dt, "unit": "convs/s", "cores": 1, "kind": "oracle", "sample": sample}
        v_all, cores, sample_all = oracle_convs_all_cores(sizes, ids, budget_s=8.0)
        cpu["all_cores"] = {"value": v_all, "unit": "convs/s", "cores": cores, "kind": "oracle",
                            "sample": sample_all}

    suite = None
    per_size = None
    if not args.no_suite and rank == 0 and world == 1:
        del hf, hg, hout
        suite = run_suite(args)
        # each size of the set alone (about 16 M elements, default plan):
        # ps per element against the HBM floor of 24 B per element
        from paper_1008_1366_gb300 import synthetic as _syn
        recs = per_size_rates(_syn.SIZES_31, reps=5, warm=3)
        per_size = {"ps_per_element": {str(r["m"]): round(r["ps_per_element"], 2) for r in recs},
                    "hbm_floor_ps_per_element": round(24.0 / measured_peak_hbm()[0] * 1e3, 2),
                    "what": "one size per launch, about 16.8 M elements, default plan (no autotuning)"}

    alg_bytes = 3 * total * 8
    avg_ms = statistics.mean(per)
    achieved = alg_bytes / (avg_ms / 1e3) / 1e9
    peak, peak_kind = measured_peak_hbm()
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": committed_traffic(alg_bytes), "peak_source": peak_kind,
            "kernel": "dc::fx::f32::fx_kernel<0> (complex kind, persistent task queue)",
            "alg_bytes_per_launch": alg_bytes}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "convs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.instances == N_INST else WORKLOAD.replace("4096", str(args.instances)),
                       "global_instances": len(sizes), "instances_rank0": n_inst, "total_elements_rank0": total,
                       "seed": SEED, "l2": "inputs larger than L2 (%.2f GB per step)" % (alg_bytes / 1e9),
                       "parallelism": (f"{world} ranks, one batch split by longest-processing-time partition "
                                       f"(cost m log2 m), no collective on the data path"),
                       "partition_max_over_mean_load": max(loads) / (sum(loads) / world),
                       "schedule": {"batch_target_tiles": plan.schedule()[0], "l1_placement": plan.schedule()[1],
                                    "task_units": plan.task_units(), "split_variant_mask": plan.variants(),
                                    "two_level_splits": {str(d[0]): "%dx%d" % (d[3], d[4])
                                                         for d in plan.describe() if d[1] == 2}}},
            "roofline": roof,
            "step_ms_stats": {"mean": T_mean, "sigma_L": sig_l, "sigma_H": sig_h, "median": statistics.median(per)},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "convs/s", "h2d_bytes_per_step": 2 * total * 8,
                    "d2h_bytes_per_step": total * 8, "chunks": e2e_chunks,
                    "api": "dc_conv_complex_1d_batched_host", "result_equals_device_path": e2e_ok},
            "clocks": clk.summary(),
            "gpu_launches": args.steps * plan.launches,
            "parity": {"max_rel_l2_sampled": worst, "worst_err_over_tol": worst_ratio,
                       "worst_pointwise_over_bar": worst_pw, "tol": "5e-7*log2(2m)", "instances_checked": len(pick),
                       "graph_replay_equals_eager": replay_ok},
            "fp64_plain": fp64,
            "cufft_padded_context": cufft,
            "trace": trace,
            "suite": suite,
            "per_size": per_size,
        }
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    if not replay_ok or not e2e_ok or worst_ratio > 1.0 or worst_pw > 1.0:
        sys.exit("parity failed: graph replay %s, e2e %s, worst rel/tol %.3g, pointwise %.3g"
                 % (replay_ok, e2e_ok, worst_ratio, worst_pw))


if __name__ == "__main__":
    main()

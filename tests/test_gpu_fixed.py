"""GPU parity of the fixed-shape engine (batched plans whose sizes all lie in
{2^a, 3*2^a, 5*2^a}, 64 <= m <= 65536; FP32 and FP64 builds) against the FP64
oracle, through the C ABI.

Covers every size of the set (both levels, every radix), partial level-1
groups, level-2 instances spread over more batches than there are scratch
regions (so regions are reused behind the dependency counters), the
pipeline-distance settings the autotuner picks from, and the status word
after each launch.  Bars per instance: relative L2 <= 5e-7 log2(2m) (FP32),
<= 1e-12 (FP64), and the pointwise bar of conftest.check_parity."""

import numpy as np
import pytest
import torch

import oracle
from conftest import FP64_TOL, check_parity, fp32_tol, norm_scale, rel_l2
from paper_1008_1366_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dc():
    import paper_1008_1366_gb300 as dc
    return dc


DTYPES = [torch.complex64, torch.complex128]


def tol(dtype, m):
    return fp32_tol(2 * m) if dtype == torch.complex64 else FP64_TOL


def run_plan(dc, sizes, seed, flags=0, dtype=torch.complex64):
    f, g, off = synthetic.batched_inputs(sizes, seed)
    plan = dc.BatchedPlan(sizes, dtype=dtype, flags=flags)
    tf = torch.tensor(f, dtype=dtype, device="cuda")
    tg = torch.tensor(g, dtype=dtype, device="cuda")
    work = plan.workspace(tf.device)
    h = plan(tf, tg, work=work)
    torch.cuda.synchronize()
    assert dc.read_status(work) == (0, 0)
    return plan, f, g, off, h.cpu().numpy()


def check_all(sizes, f, g, off, h, dtype=torch.complex64):
    worst = 0.0
    for i, m in enumerate(sizes):
        a, b = off[i], off[i + 1]
        ref = oracle.padded_complex(f[a:b], g[a:b])
        e, _ = check_parity(h[a:b], ref, dtype, 2 * m, norm_scale(f[a:b], g[a:b]), what=f"instance {i} m={m}")
        worst = max(worst, e / tol(dtype, m))
    return worst


@pytest.mark.parametrize("dtype", DTYPES)
def test_every_size_once(dc, dtype):
    sizes = list(synthetic.SIZES_31)
    plan, f, g, off, h = run_plan(dc, sizes, 21, dtype=dtype)
    assert plan.launches == 1
    desc = plan.describe()
    assert sorted(d[0] for d in desc) == sorted(sizes)
    levels = {d[0]: d[1] for d in desc}
    assert levels[64] == 1 and levels[96] == 1 and levels[80] == 1
    assert levels[16384] == 2 and levels[65536] == 2 and levels[20480] == 2 and levels[24576] == 2
    # within a size family the level never drops as m grows
    for base in (64, 96, 80):
        fam = sorted(m for m in sizes if m % base == 0 and (m // base) & (m // base - 1) == 0)
        lv = [levels[m] for m in fam]
        assert lv == sorted(lv)
    check_all(sizes, f, g, off, h, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_partial_groups_and_order(dc, dtype):
    # level-1 groups that are full, partial and single; sizes interleaved
    sizes = [64] * 130 + [96] * 3 + [4096] * 3 + [80, 160, 320] * 5 + [8192, 12288, 10240] * 2
    rng = np.random.default_rng(3)
    sizes = [sizes[i] for i in rng.permutation(len(sizes))]
    _, f, g, off, h = run_plan(dc, sizes, 22, dtype=dtype)
    check_all(sizes, f, g, off, h, dtype)


def test_trace_counts_every_task(dc):
    # the header's trace counts one entry per task of the queue
    sizes = [65536] * 2 + [640] * 20 + [64] * 130
    plan, f, g, off, h = run_plan(dc, sizes, 29)
    tr = dc.read_trace(plan.workspace(torch.device("cuda")))
    # 65536 = 256 x 256: 16 column tiles (A and C) and 32 row groups (B) each
    assert tr["tasks"] == {"L1": 3 + 3, "A": 32, "B": 64, "C": 32}, tr
    assert all(v > 0 for v in tr["cycles"].values())


@pytest.mark.parametrize("dtype", DTYPES)
def test_level2_region_reuse(dc, dtype):
    # many level-2 instances: more batches than the four scratch regions
    sizes = [65536] * 24 + [16384] * 30 + [49152] * 6 + [20480] * 8 + [2048] * 20
    rng = np.random.default_rng(4)
    sizes = [sizes[i] for i in rng.permutation(len(sizes))]
    _, f, g, off, h = run_plan(dc, sizes, 23, dtype=dtype)
    check_all(sizes, f, g, off, h, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_one_per_launch(dc, dtype):
    # the plain mode: one launch per instance, each over its own task range
    sizes = [65536, 64, 12288, 640, 40960, 96, 4096]
    plan, f, g, off, h = run_plan(dc, sizes, 28, flags=4, dtype=dtype)
    assert plan.launches == len(sizes)
    assert plan.schedule() is None
    check_all(sizes, f, g, off, h, dtype)


def test_autotuned_plan_matches(dc):
    sizes = [65536] * 6 + [40960] * 4 + [640] * 40 + [24576] * 4
    plan, f, g, off, h = run_plan(dc, sizes, 24, flags=1)
    check_all(sizes, f, g, off, h)


def test_repeat_launch_same_result(dc):
    # counters and the queue are reset per launch: a second launch on the
    # same workspace reproduces the first bit for bit
    sizes = [32768] * 5 + [1536] * 9 + [5120] * 3
    f, g, off = synthetic.batched_inputs(sizes, 25)
    plan = dc.BatchedPlan(sizes, dtype=torch.complex64)
    tf = torch.tensor(f, dtype=torch.complex64, device="cuda")
    tg = torch.tensor(g, dtype=torch.complex64, device="cuda")
    work = plan.workspace(tf.device)
    h1 = plan(tf, tg, work=work).clone()
    h2 = plan(tf, tg, work=work)
    torch.cuda.synchronize()
    assert torch.equal(h1, h2)
    check_all(sizes, f, g, off, h2.cpu().numpy())


def test_special_inputs(dc):
    # delta inputs: f = e_0 gives h = g exactly up to rounding
    sizes = [64, 12288, 65536]
    total = sum(sizes)
    rng = np.random.default_rng(7)
    g = (rng.uniform(-1, 1, total) + 1j * rng.uniform(-1, 1, total))
    f = np.zeros(total, dtype=np.complex128)
    off = np.concatenate([[0], np.cumsum(sizes)])
    for i in range(len(sizes)):
        f[off[i]] = 1.0
    plan = dc.BatchedPlan(sizes, dtype=torch.complex64)
    tf = torch.tensor(f, dtype=torch.complex64, device="cuda")
    tg = torch.tensor(g, dtype=torch.complex64, device="cuda")
    h = plan(tf, tg).cpu().numpy()
    for i, m in enumerate(sizes):
        a, b = off[i], off[i + 1]
        check_parity(h[a:b], g[a:b], torch.complex64, 2 * m, norm_scale(f[a:b], g[a:b]))


def test_schedules_give_identical_results(dc):
    # the queue order changes timing only: every schedule gives the same bits
    sizes = [65536] * 3 + [24576] * 4 + [640] * 30 + [64] * 70 + [12288] * 2
    f, g, off = synthetic.batched_inputs(sizes, 26)
    plan = dc.BatchedPlan(sizes, dtype=torch.complex64)
    assert plan.schedule() is not None
    tf = torch.tensor(f, dtype=torch.complex64, device="cuda")
    tg = torch.tensor(g, dtype=torch.complex64, device="cuda")
    ref = plan(tf, tg).clone()
    for target in (1, 7, 152):
        for mode in (0, 1, 2):
            for units in (1, 2, 4):
                plan.set_task_units(units)
                plan.set_schedule(target, mode)
                assert plan.schedule() == (target, mode) and plan.task_units() == units
                work = plan.workspace(tf.device)
                h = plan(tf, tg, work=work)
                torch.cuda.synchronize()
                assert dc.read_status(work) == (0, 0)
                assert torch.equal(h, ref), (target, mode, units)
    check_all(sizes, f, g, off, ref.cpu().numpy())
    other = dc.BatchedPlan(sizes + [48], dtype=torch.complex64)   # 48 < 64: runtime-shaped engine
    assert other.schedule() is None and other.task_units() is None
    from paper_1008_1366_gb300 import api
    with pytest.raises(api.DealiasError):
        plan.set_task_units(5)


@pytest.mark.parametrize("dtype", DTYPES)
def test_task_units_for_every_mode(dc, dtype):
    # several tiles or row groups per task: the trace counts units of work
    # once per task, and the result does not change
    sizes = [65536] * 2 + [640] * 20 + [64] * 130
    plan, f, g, off, h1 = run_plan(dc, sizes, 36, dtype=dtype)
    plan.set_task_units(4)
    tf = torch.tensor(f, dtype=dtype, device="cuda")
    tg = torch.tensor(g, dtype=dtype, device="cuda")
    work = plan.workspace(tf.device)
    h4 = plan(tf, tg, work=work)
    torch.cuda.synchronize()
    assert dc.read_status(work) == (0, 0)
    assert np.array_equal(h4.cpu().numpy(), h1)
    tr = dc.read_trace(work)
    assert tr["tasks"] == {"L1": 3 + 3, "A": 8, "B": 16, "C": 8}, tr
    check_all(sizes, f, g, off, h1, dtype)


def test_bounded_wait_reports_timeout(dc):
    # a dependency nothing satisfies: the kernel's bounded wait runs out
    # after about a millisecond, records DC_ERR_TIMEOUT and the launch ends
    import ctypes
    from paper_1008_1366_gb300 import _native
    L = _native.lib()
    work = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.dc_selftest_wait_timeout(ctypes.c_void_p(work.data_ptr()), work.numel(), 2_000_000, s) == 0
    torch.cuda.synchronize()
    assert dc.read_status(work) == (5, 0)
    # the context stays usable: an ordinary plan runs and is correct
    sizes = [64, 65536]
    _, f, g, off, h = run_plan(dc, sizes, 27)
    check_all(sizes, f, g, off, h)
    # argument checks
    assert L.dc_selftest_wait_timeout(ctypes.c_void_p(work.data_ptr()), 100, 1000, s) == 6
    assert L.dc_selftest_wait_timeout(ctypes.c_void_p(work.data_ptr() + 8), 4000, 1000, s) == 3
    assert L.dc_selftest_wait_timeout(ctypes.c_void_p(0), 4096, 1000, s) == 1


@pytest.mark.parametrize("nchunks", [1, 3, 8])
def test_host_pipeline_matches(dc, nchunks):
    # host-to-host pipelined execution gives the device path's bits
    sizes = list(synthetic.batched_sizes(200, 31))
    f, g, off = synthetic.batched_inputs(sizes, 30)
    plan = dc.BatchedPlan(sizes, dtype=torch.complex64)
    df = torch.tensor(f, dtype=torch.complex64, device="cuda")
    dg = torch.tensor(g, dtype=torch.complex64, device="cuda")
    ref = plan(df, dg).cpu()
    hf = torch.tensor(f, dtype=torch.complex64).pin_memory()
    hg = torch.tensor(g, dtype=torch.complex64).pin_memory()
    hh = torch.zeros_like(hf).pin_memory()
    dh = torch.empty_like(df)
    df.zero_()
    dg.zero_()
    work = plan.host_workspace(nchunks, df.device)
    plan.run_from_host(hf, hg, hh, df, dg, dh, work, nchunks)
    torch.cuda.synchronize()
    assert torch.equal(hh, ref)


def test_host_pipeline_runtime_engine(dc):
    # also for plans on the runtime-shaped engine (a size outside the set)
    sizes = [48, 1024, 7 * 0 + 6, 3072, 96]
    f, g, off = synthetic.batched_inputs(sizes, 32)
    plan = dc.BatchedPlan(sizes, dtype=torch.complex128)
    hf = torch.tensor(f, dtype=torch.complex128).pin_memory()
    hg = torch.tensor(g, dtype=torch.complex128).pin_memory()
    hh = torch.zeros_like(hf).pin_memory()
    df, dg, dh = (torch.empty(hf.numel(), dtype=torch.complex128, device="cuda") for _ in range(3))
    work = plan.host_workspace(2, df.device)
    plan.run_from_host(hf, hg, hh, df, dg, dh, work, 2)
    torch.cuda.synchronize()
    check_all(sizes, f, g, off, hh.numpy(), torch.complex128)


@pytest.mark.parametrize("dtype", DTYPES)
def test_in_place(dc, dtype):
    # h may be f or g: every instance reads its inputs before writing h
    sizes = [64, 640, 4096, 12288, 65536, 96] * 3
    f, g, off = synthetic.batched_inputs(sizes, 33)
    plan = dc.BatchedPlan(sizes, dtype=dtype)
    for target in ("f", "g"):
        tf = torch.tensor(f, dtype=dtype, device="cuda")
        tg = torch.tensor(g, dtype=dtype, device="cuda")
        out = tf if target == "f" else tg
        plan(tf, tg, out=out)
        torch.cuda.synchronize()
        check_all(sizes, f, g, off, out.cpu().numpy(), dtype)


def test_graph_replay_matches_eager_and_oracle(dc):
    # the benchmark's form of the call: one persistent launch captured in a
    # CUDA graph.  Replays give the eager launch's bits, and a replay after
    # the inputs change in place convolves the new inputs.
    sizes = [65536] * 2 + [12288] * 3 + [40960] + [640] * 20 + [64] * 40 + [96] * 9
    f, g, off = synthetic.batched_inputs(sizes, 34)
    f2, g2, _ = synthetic.batched_inputs(sizes, 35)
    plan = dc.BatchedPlan(sizes, dtype=torch.complex64)
    tf = torch.tensor(f, dtype=torch.complex64, device="cuda")
    tg = torch.tensor(g, dtype=torch.complex64, device="cuda")
    out = torch.empty_like(tf)
    work = plan.workspace(tf.device)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan(tf, tg, out=out, work=work)
    s.synchronize()
    eager = out.clone()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        plan(tf, tg, out=out, work=work)
    for _ in range(2):
        out.zero_()
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        assert dc.read_status(work) == (0, 0)
        assert torch.equal(out, eager)
    check_all(sizes, f, g, off, out.cpu().numpy())
    tf.copy_(torch.tensor(f2, dtype=torch.complex64))
    tg.copy_(torch.tensor(g2, dtype=torch.complex64))
    torch.cuda.synchronize()
    graph.replay()
    torch.cuda.synchronize()
    check_all(sizes, f2, g2, off, out.cpu().numpy())


TWO_LEVEL = [8192, 16384, 32768, 65536, 12288, 24576, 49152, 10240, 20480, 40960]


def size_code_of(m):
    # the engine's size codes: 64 << c (c < 11), 96 << (c - 11), 80 << (c - 21)
    for c, base in ((0, 64), (11, 96), (21, 80)):
        k = m // base
        if m % base == 0 and k & (k - 1) == 0:
            return c + k.bit_length() - 1
    raise ValueError(m)


def test_split_variants_every_two_level_size(dc):
    # variant 1 of the two-level split (L2 = 64 for the smallest two-level
    # size of each family, else 256 up to m = 32768 and 128 above): every
    # two-level size, several instances each, against the
    # oracle; describe reports the swapped split and the mask reads back
    sizes = [m for m in TWO_LEVEL for _ in range(3)] + [640] * 20 + [64] * 70
    rng = np.random.default_rng(41)
    sizes = [sizes[i] for i in rng.permutation(len(sizes))]
    f, g, off = synthetic.batched_inputs(sizes, 41)
    plan = dc.BatchedPlan(sizes, dtype=torch.complex64)
    assert plan.variants() == 0
    before = {d[0]: d for d in plan.describe()}
    full = sum(1 << size_code_of(m) for m in TWO_LEVEL)
    plan.set_variants(0xFFFFFFFF)
    assert plan.variants() == full
    after = {d[0]: d for d in plan.describe()}
    for m in TWO_LEVEL:
        l1, l2 = before[m][3], before[m][4]
        assert l1 * l2 == m and after[m][3] * after[m][4] == m
        want = 64 if m in (8192, 12288, 10240) else (256 if l2 == 128 else 128)
        assert after[m][4] == want, (m, before[m], after[m])
    assert after[640] == before[640] and after[64] == before[64]
    tf = torch.tensor(f, dtype=torch.complex64, device="cuda")
    tg = torch.tensor(g, dtype=torch.complex64, device="cuda")
    work = plan.workspace(tf.device)
    h = plan(tf, tg, work=work)
    torch.cuda.synchronize()
    assert dc.read_status(work) == (0, 0)
    check_all(sizes, f, g, off, h.cpu().numpy())


def test_split_variant_masks_and_schedules(dc):
    # alternating masks, with the pipeline settings: every combination gives
    # a correct result, and the level-1 work is untouched by the mask
    sizes = [65536] * 3 + [10240] * 5 + [24576] * 4 + [8192] * 6 + [1280] * 12 + [96] * 40
    f, g, off = synthetic.batched_inputs(sizes, 42)
    plan = dc.BatchedPlan(sizes, dtype=torch.complex64)
    tf = torch.tensor(f, dtype=torch.complex64, device="cuda")
    tg = torch.tensor(g, dtype=torch.complex64, device="cuda")
    codes = [size_code_of(m) for m in (65536, 10240, 24576, 8192)]
    for mask in ((1 << codes[0]) | (1 << codes[2]), (1 << codes[1]) | (1 << codes[3]), sum(1 << c for c in codes)):
        for target, mode, units in ((1, 0, 1), (152, 1, 2), (38, 2, 4)):
            plan.set_variants(mask)
            plan.set_task_units(units)
            plan.set_schedule(target, mode)
            assert plan.variants() == mask
            work = plan.workspace(tf.device)
            h = plan(tf, tg, work=work)
            torch.cuda.synchronize()
            assert dc.read_status(work) == (0, 0)
            check_all(sizes, f, g, off, h.cpu().numpy())


def test_split_variants_fp64_ignored(dc):
    # FP64 plans run variant 0 only: the mask is accepted and dropped
    sizes = [16384] * 2 + [640] * 4
    plan = dc.BatchedPlan(sizes, dtype=torch.complex128)
    plan.set_variants(0xFFFFFFFF)
    assert plan.variants() == 0
    _, f, g, off, h = run_plan(dc, sizes, 43, dtype=torch.complex128)
    check_all(sizes, f, g, off, h, torch.complex128)


def test_autotuned_variants_valid(dc):
    # the autotuner's choice is a subset of the sizes that have a second
    # split, and the tuned plan is correct
    sizes = [m for m in TWO_LEVEL for _ in range(4)] + [640] * 40
    plan, f, g, off, h = run_plan(dc, sizes, 44, flags=1)
    full = sum(1 << size_code_of(m) for m in TWO_LEVEL)
    v = plan.variants()
    assert v is not None and (v & ~full) == 0
    check_all(sizes, f, g, off, h)


def test_host_pipeline_follows_variants(dc):
    # the host-to-host pipeline's chunk plans run the plan's split variants,
    # so its result stays the device path's bits when the variants change
    sizes = [65536] * 2 + [10240] * 4 + [12288] * 3 + [640] * 30
    f, g, off = synthetic.batched_inputs(sizes, 45)
    plan = dc.BatchedPlan(sizes, dtype=torch.complex64)
    df0 = torch.tensor(f, dtype=torch.complex64, device="cuda")
    dg0 = torch.tensor(g, dtype=torch.complex64, device="cuda")
    hf = torch.tensor(f, dtype=torch.complex64).pin_memory()
    hg = torch.tensor(g, dtype=torch.complex64).pin_memory()
    for mask in (0, 0xFFFFFFFF, 1 << size_code_of(10240)):
        plan.set_variants(mask)
        ref = plan(df0, dg0).cpu()
        hh = torch.zeros_like(hf).pin_memory()
        df, dg, dh = (torch.empty_like(df0) for _ in range(3))
        work = plan.host_workspace(3, df.device)
        plan.run_from_host(hf, hg, hh, df, dg, dh, work, 3)
        torch.cuda.synchronize()
        assert torch.equal(hh, ref), hex(mask)
        check_all(sizes, f, g, off, hh.numpy())

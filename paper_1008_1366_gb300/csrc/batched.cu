// Batched 1D complex convolutions of uneven sizes in one persistent launch.
//
// Batches whose sizes all lie in the set {2^a, 3*2^a, 5*2^a} in [64, 65536]
// run on the fixed-shape engine (fixed.cuh, fixed_batched.cu; FP32 and FP64
// builds): a task queue of level-1 groups and level-2 pass tasks, one launch
// (or, in the plain mode, one launch per instance).  Other batches run on
// the runtime-shaped engine (conv1d.cuh), as follows.
//
// Planning groups the instances by size; each size gets a configuration
// (level 1: `nt` instances per block wholly in shared memory; level 2: one
// instance per block through a scratch slot).  With DC_PLAN_AUTOTUNE the
// configuration of every size is chosen by timing the candidates of
// enumerate_cfgs on the device, on that size's own instance count.  Work
// items (a group of same-size instances, or one large instance) are sorted
// by estimated cost, largest first, and a persistent grid of
// (SMs x resident blocks) takes them from an atomic counter, which balances
// uneven sizes like a longest-processing-time schedule.
#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

#include "conv1d.cuh"
#include "fixed.h"
#include "launch.h"
#include "plan.h"
#include "tables.h"

using namespace dc;

struct dc_batched_plan {
  int32_t dtype = 0, ds = 0, flags = 0, n = 0;
  int64_t total = 0;
  int device = 0;
  std::vector<CfgDev> cfgs;
  std::vector<Item> items;
  char* dmem = nullptr;       // one device allocation: cfgs, items, order, offsets
  CfgDev* d_cfgs = nullptr;
  Item* d_items = nullptr;
  int32_t* d_order = nullptr;
  int64_t* d_off = nullptr;
  int grid = 0, smem = 0;
  size_t slot = 0, work = 0;
  // fixed-shape engine
  bool fx = false;
  int mode = fx::MODE_COMPLEX;   // kind of convolution (fx::MODE_*; others internal plans only)
  const struct FxOps* ops = nullptr;
  fx::HostPlan hp;
  fx::Task* d_tasks = nullptr;
  fx::L2Inst* d_l2 = nullptr;
  int64_t* d_l1tmp = nullptr;
  const void* tabs[fx::kNumCodes] = {};    // root tables per kernel code
  const void* stabs[fx::kNumCodes] = {};   // stage-twiddle tables (null: none)
  size_t cnt_bytes = 0;   // header + counters, zeroed before each launch
  fx::Schedule fx_sched{0, 0};   // queue order of the fixed engine
  std::vector<int64_t> off_host;
  // plain mode: one launch per instance over its own task range
  std::vector<int32_t> inst_first, inst_count;
  // pipelined host-to-host execution: chunk plans over consecutive instances
  struct Chunks {
    int n = 0;
    std::vector<dc_batched_plan*> plans;
    std::vector<int32_t> first;      // first instance of each chunk
    size_t work = 0;                 // shared workspace of the chunk plans
    cudaStream_t st[4] = {nullptr, nullptr, nullptr, nullptr};   // copy f in, compute, copy out, copy g in
    std::vector<cudaEvent_t> ev;     // per chunk: f arrived, results ready, g arrived; then 5 joins
  } chunks;
  std::vector<int64_t> m_host;
};

// one precision of the fixed-shape engine
struct FxOps {
  int (*size_code)(int64_t);
  int64_t (*code_size)(int);
  void (*code_shape)(int, int*, int*, int*, int*, int*);
  int (*code_smem)(int);
  bool (*build_plan)(const int64_t*, int32_t, const int64_t*, const fx::Schedule&, int, fx::HostPlan*);
  dc_status (*prepare_kernel)(int, int*);
  dc_status (*launch)(const fx::FxArgs&, int, int, cudaStream_t);
  void (*code_tabs)(int, int*, int*);
  dc_status (*stage_tables)(int, const void**);
  bool (*code_ok)(int, int);
};
static const FxOps kFx32{fx::f32::size_code,      fx::f32::code_size,  fx::f32::code_shape, fx::f32::code_smem,
                         fx::f32::build_plan,     fx::f32::prepare_kernel, fx::f32::launch, fx::f32::code_tabs,
                         fx::f32::stage_tables, fx::f32::code_ok};
static const FxOps kFx64{fx::f64::size_code,      fx::f64::code_size,  fx::f64::code_shape, fx::f64::code_smem,
                         fx::f64::build_plan,     fx::f64::prepare_kernel, fx::f64::launch, fx::f64::code_tabs,
                         fx::f64::stage_tables, fx::f64::code_ok};

namespace {
size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// The largest dynamic shared memory of any kernel code of a precision: the
// kernels' attribute is set to it everywhere, so that no caller lowers it
// below what another plan launches with.
int fx_smem_all(const FxOps* ops) {
  int smem = 0;
  for (int c = 0; c < fx::kNumCodes; ++c)
    if (ops->code_ok(c, fx::MODE_COMPLEX)) smem = std::max(smem, ops->code_smem(c));
  return smem;
}

double item_cost(const CfgDev& c, int count) {
  // six sub-transforms of length L per instance plus the level-2 passes
  double f = 6.0 * (double)std::max<int64_t>(fft_flops(c.L), c.L) * count;
  if (c.level == 2) f *= 1.5;
  return f;
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
};

// Times one configuration on `count` instances of size m: persistent launch
// over the instances' items, median of three runs (ms); < 0 on failure.
float time_cfg(const CfgDev& c, int count, int ds, const void* f, const void* g, void* h, cudaStream_t s) {
  std::vector<Item> items;
  const int per = c.level == 1 ? c.nt : 1;
  for (int i = 0; i < count; i += per) items.push_back(Item{0, i, std::min(per, count - i), 0});
  int bps = 1;
  if (conv1d_blocks_per_sm(K_COMPLEX, ds, c.smem, &bps) != DC_OK || bps < 1) return -1;
  const int grid = bps * device_info().sms;
  const size_t slot = align_up(cfg_scratch_bytes(K_COMPLEX, c, ds), 256);
  DevBuf dcfg, ditems, dwork;
  if (cudaMalloc(&dcfg.p, sizeof(CfgDev)) != cudaSuccess) return -1;
  if (cudaMalloc(&ditems.p, items.size() * sizeof(Item)) != cudaSuccess) return -1;
  if (cudaMalloc(&dwork.p, sizeof(WorkHeader) + (size_t)grid * slot) != cudaSuccess) return -1;
  cudaMemcpy(dcfg.p, &c, sizeof(CfgDev), cudaMemcpyHostToDevice);
  cudaMemcpy(ditems.p, items.data(), items.size() * sizeof(Item), cudaMemcpyHostToDevice);
  ConvArgs a{};
  a.in[0] = f;
  a.in[1] = g;
  a.out[0] = h;
  a.stride = c.m;
  a.items = (const Item*)ditems.p;
  a.nitems = (int32_t)items.size();
  a.ninst = count;
  a.cfgs = (const CfgDev*)dcfg.p;
  a.hdr = (WorkHeader*)dwork.p;
  a.scratch = (char*)dwork.p + sizeof(WorkHeader);
  a.slot_bytes = (int64_t)slot;
  a.persistent = 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<float> t;
  for (int rep = 0; rep < 4; ++rep) {
    cudaMemsetAsync(dwork.p, 0, sizeof(WorkHeader), s);
    cudaEventRecord(e0, s);
    if (launch_conv1d(K_COMPLEX, ds, a, grid, c.smem, s) != DC_OK) break;
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) t.push_back(ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess || t.size() < 3) return -1;
  std::sort(t.begin(), t.end());
  return t[1];
}

dc_status autotune_size(int64_t m, int count, int ds, int smem_max, CfgDev* best) {
  CfgDev cands[24];
  const int nc = enumerate_cfgs(K_COMPLEX, m, ds, kThreads, smem_max, cands, 24);
  if (nc <= 1) return DC_OK;
  const int cnt = std::max(1, std::min(count, 4096));
  const size_t bytes = (size_t)cnt * m * ds;
  DevBuf f, g, h;
  DC_CUDA_TRY(cudaMalloc(&f.p, bytes));
  DC_CUDA_TRY(cudaMalloc(&g.p, bytes));
  DC_CUDA_TRY(cudaMalloc(&h.p, bytes));
  DC_CUDA_TRY(cudaMemset(f.p, 0x3c, bytes));   // finite, normal values
  DC_CUDA_TRY(cudaMemset(g.p, 0x3b, bytes));
  cudaStream_t s;
  DC_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  float tbest = -1;
  for (int k = 0; k < nc; ++k) {
    const void* tw = nullptr;
    if (get_root_table(cands[k].TN, ds, &tw) != DC_OK) continue;
    cands[k].tw = tw;
    const float t = time_cfg(cands[k], cnt, ds, f.p, g.p, h.p, s);
    if (t > 0 && (tbest < 0 || t < tbest)) { tbest = t; *best = cands[k]; }
  }
  cudaStreamDestroy(s);
  cudaGetLastError();
  return DC_OK;
}
// workspace: header + counters | level-2 scratch | level-1 partial outputs
size_t fx_tmp_offset(const dc_batched_plan* p) {
  return p->cnt_bytes + align_up(p->hp.scratch * (size_t)p->ds, 256);
}
size_t fx_work_bytes(const dc_batched_plan* p) {
  return fx_tmp_offset(p) + p->hp.l1_elems * (size_t)p->ds;
}

dc_status fx_upload(dc_batched_plan* p, const std::vector<int64_t>& off) {
  if (p->dmem) { cudaFree(p->dmem); p->dmem = nullptr; }
  const fx::HostPlan& hp = p->hp;
  const size_t bt = align_up(std::max<size_t>(1, hp.tasks.size()) * sizeof(fx::Task), 256);
  const size_t bl = align_up(std::max<size_t>(1, hp.l2.size()) * sizeof(fx::L2Inst), 256);
  const size_t bo = align_up(std::max<size_t>(1, hp.order.size()) * sizeof(int32_t), 256);
  const size_t bf = align_up(off.size() * sizeof(int64_t), 256);
  const size_t bp = align_up(std::max<size_t>(1, hp.l1tmp.size()) * sizeof(int64_t), 256);
  DC_CUDA_TRY(cudaMalloc(&p->dmem, bt + bl + bo + bf + bp));
  p->d_tasks = (fx::Task*)p->dmem;
  p->d_l2 = (fx::L2Inst*)(p->dmem + bt);
  p->d_order = (int32_t*)(p->dmem + bt + bl);
  p->d_off = (int64_t*)(p->dmem + bt + bl + bo);
  p->d_l1tmp = (int64_t*)(p->dmem + bt + bl + bo + bf);
  if (!hp.l1tmp.empty())
    DC_CUDA_TRY(cudaMemcpy(p->d_l1tmp, hp.l1tmp.data(), hp.l1tmp.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  if (!hp.tasks.empty())
    DC_CUDA_TRY(cudaMemcpy(p->d_tasks, hp.tasks.data(), hp.tasks.size() * sizeof(fx::Task), cudaMemcpyHostToDevice));
  if (!hp.l2.empty())
    DC_CUDA_TRY(cudaMemcpy(p->d_l2, hp.l2.data(), hp.l2.size() * sizeof(fx::L2Inst), cudaMemcpyHostToDevice));
  if (!hp.order.empty())
    DC_CUDA_TRY(cudaMemcpy(p->d_order, hp.order.data(), hp.order.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  DC_CUDA_TRY(cudaMemcpy(p->d_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  p->cnt_bytes = align_up(sizeof(WorkHeader) + hp.ncnt * sizeof(uint32_t), 256);
  p->work = fx_work_bytes(p);
  p->smem = hp.smem;
  return DC_OK;
}

// root and stage-twiddle tables of every kernel code of the plan's queue
dc_status fx_tables(dc_batched_plan* p) {
  for (int c : p->hp.codes) {
    if (!p->tabs[c]) {
      dc_status st = get_root_table(fx::mode_q(p->mode) * p->ops->code_size(c), p->ds, &p->tabs[c]);
      if (st != DC_OK) return st;
    }
    if (!p->stabs[c]) {
      dc_status st = p->ops->stage_tables(c, &p->stabs[c]);
      if (st != DC_OK) return st;
    }
  }
  return DC_OK;
}

// rebuilds the queue of plan p in schedule sc (tables, upload)
dc_status fx_rebuild(dc_batched_plan* p, const int64_t* m, int32_t n, const std::vector<int64_t>& off,
                     const fx::Schedule& sc) {
  if (!p->ops->build_plan(m, n, off.data(), sc, p->mode, &p->hp)) return DC_ERR_SIZE;
  dc_status st = fx_tables(p);
  if (st != DC_OK) return st;
  return fx_upload(p, off);
}

fx::FxArgs fx_args(const dc_batched_plan* p, const void* f, const void* g, void* h, void* work,
                   const void* e = nullptr, void* h2 = nullptr, const void* e2 = nullptr) {
  fx::FxArgs a{};
  a.f = f;
  a.g = g;
  a.h = h;
  a.e = e;
  a.e2 = e2;
  a.h2 = h2;
  a.mode = p->mode;
  a.off = p->d_off;
  a.order = p->d_order;
  a.tasks = p->d_tasks;
  a.ntasks = (int32_t)p->hp.tasks.size();
  a.l2 = p->d_l2;
  a.hdr = (WorkHeader*)work;
  a.cnt = (uint32_t*)((char*)work + sizeof(WorkHeader));
  a.scratch = (char*)work + p->cnt_bytes;
  a.tmp = (char*)work + fx_tmp_offset(p);
  a.l1tmp = p->d_l1tmp;
  auto aliases = [&](const void* o) { return o && (o == f || o == g || o == e || o == e2); };
  a.in_place = (aliases(h) || aliases(h2)) ? 1 : 0;
  a.wait_limit = fx::kWaitLimit;
  for (int c = 0; c < fx::kNumCodes; ++c) {
    a.tab[c] = p->tabs[c];
    a.stab[c] = p->stabs[c];
    if (p->stabs[c]) p->ops->code_tabs(c, &a.stab_n[c], &a.stab_off[c]);
  }
  return a;
}

dc_status fx_launch(const dc_batched_plan* p, const void* f, const void* g, void* h, void* work, cudaStream_t s,
                    const void* e = nullptr, void* h2 = nullptr, const void* e2 = nullptr) {
  DC_CUDA_TRY(cudaMemsetAsync(work, 0, p->cnt_bytes, s));
  fx::FxArgs a = fx_args(p, f, g, h, work, e, h2, e2);
  if (p->inst_first.empty()) return p->ops->launch(a, p->grid, p->smem, s);
  // plain mode: each instance's tasks in a launch of their own (the queue
  // counter is reset before each; the dependency counters are distinct)
  const fx::Task* base = a.tasks;
  for (size_t i = 0; i < p->inst_first.size(); ++i) {
    if (i > 0) DC_CUDA_TRY(cudaMemsetAsync(&((WorkHeader*)work)->counter, 0, sizeof(uint32_t), s));
    a.tasks = base + p->inst_first[i];
    a.ntasks = p->inst_count[i];
    dc_status st = p->ops->launch(a, std::min(p->grid, (int)a.ntasks), p->smem, s);
    if (st != DC_OK) return st;
  }
  return DC_OK;
}

// Times the whole batch on scratch buffers (median of three after a warm-up, ms).
// median time of a launch of plan p (one untimed launch, then `reps`)
float fx_time(dc_batched_plan* p, cudaStream_t s, int reps = 3) {
  DevBuf f, g, h, w;
  const size_t bytes = (size_t)p->total * (size_t)p->ds;
  if (cudaMalloc(&f.p, bytes) != cudaSuccess || cudaMalloc(&g.p, bytes) != cudaSuccess ||
      cudaMalloc(&h.p, bytes) != cudaSuccess || cudaMalloc(&w.p, p->work) != cudaSuccess)
    return -1;
  cudaMemset(f.p, 0x3c, bytes);
  cudaMemset(g.p, 0x3b, bytes);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<float> t;
  for (int rep = 0; rep <= reps; ++rep) {
    cudaEventRecord(e0, s);
    if (fx_launch(p, f.p, g.p, h.p, w.p, s) != DC_OK) break;
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) t.push_back(ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int32_t st[2] = {0, 0};
  cudaMemcpy(st, w.p, sizeof(st), cudaMemcpyDeviceToHost);
  if (cudaGetLastError() != cudaSuccess || (int)t.size() < reps || st[0] != 0) return -1;
  std::sort(t.begin(), t.end());
  return t[t.size() / 2];
}

// Plain mode: the queues of one-instance plans, concatenated in instance
// order, each launched on its own.  They run one after another, so they
// share one scratch region.
bool fx_build_plain(dc_batched_plan* p, const int64_t* m, int32_t n, const std::vector<int64_t>& off) {
  fx::HostPlan all;
  p->inst_first.clear();
  p->inst_count.clear();
  const fx::Schedule sc{p->grid / 2, 0};
  for (int32_t i = 0; i < n; ++i) {
    fx::HostPlan one;
    if (!p->ops->build_plan(m + i, 1, off.data() + i, sc, p->mode, &one)) return false;
    const int32_t ob = (int32_t)all.order.size(), lb = (int32_t)all.l2.size(), cb = (int32_t)all.ncnt;
    p->inst_first.push_back((int32_t)all.tasks.size());
    p->inst_count.push_back((int32_t)one.tasks.size());
    for (fx::Task t : one.tasks) {
      if (((t.kc >> 8) & 255) == fx::T_L1) t.a += ob;
      else t.a += lb;
      if (t.widx >= 0) t.widx += cb;
      if (t.sidx >= 0) t.sidx += cb;
      all.tasks.push_back(t);
    }
    for (int32_t id : one.order) all.order.push_back(id + i);   // the one-instance plan numbers it 0
    all.l2.insert(all.l2.end(), one.l2.begin(), one.l2.end());
    all.ncnt += one.ncnt;
    all.scratch = std::max(all.scratch, one.scratch);
    all.l1tmp.push_back(0);   // the launches run one after another: one shared region
    all.l1_elems = std::max(all.l1_elems, one.l1_elems);
    all.smem = std::max(all.smem, one.smem);
    for (int c : one.codes)
      if (std::find(all.codes.begin(), all.codes.end(), c) == all.codes.end()) all.codes.push_back(c);
  }
  std::sort(all.codes.begin(), all.codes.end());
  p->hp = std::move(all);
  return true;
}

dc_status create_fixed(dc_batched_plan* p, const int64_t* m, int32_t n, const std::vector<int64_t>& off,
                       int32_t flags, int mode = fx::MODE_COMPLEX) {
  p->fx = true;
  p->mode = mode;
  p->ops = p->ds == 8 ? &kFx32 : &kFx64;
  p->off_host = off;
  int bps = 0;
  // kernel attributes for the largest shared-memory need of any size
  dc_status st = p->ops->prepare_kernel(fx_smem_all(p->ops), &bps);
  if (st != DC_OK) return st;
  p->grid = bps * device_info().sms;
  const fx::Schedule dflt{p->grid / 2, 0};
  const bool plain = (flags & DC_PLAN_ONE_PER_LAUNCH) != 0;
  if (plain ? !fx_build_plain(p, m, n, off) : !p->ops->build_plan(m, n, off.data(), dflt, p->mode, &p->hp))
    return DC_ERR_SIZE;
  st = fx_tables(p);
  if (st != DC_OK) return st;
  st = fx_upload(p, off);
  if (st != DC_OK) return st;
  p->fx_sched = dflt;
  if ((flags & DC_PLAN_AUTOTUNE) && !plain) {
    cudaStream_t s;
    DC_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    // The split of each two-level size (the row and column lengths, the
    // column tile width and the threads per row follow from it): variant 0
    // or 1, timed on the instances of that size alone, kept where it is at
    // least 1 % faster.
    uint32_t vmask = 0;
    for (int c = 0; c < fx::kNumSizes; ++c) {
      if (!p->ops->code_ok(c + fx::kCodeStride, p->mode)) continue;
      std::vector<int64_t> mc, oc;
      for (int32_t i = 0; i < n; ++i)
        if (p->ops->size_code(m[i]) == c) {
          mc.push_back(m[i]);
          oc.push_back(off[i]);
        }
      if (mc.empty()) continue;
      float tv[2] = {-1, -1};
      for (int v = 0; v < 2; ++v) {
        fx::Schedule sc = dflt;
        sc.variants = (uint32_t)v << c;
        // short launches: more repetitions for a stable median
        if (fx_rebuild(p, mc.data(), (int32_t)mc.size(), oc, sc) == DC_OK) tv[v] = fx_time(p, s, 9);
      }
      if (tv[0] > 0 && tv[1] > 0 && tv[1] < 0.99f * tv[0]) vmask |= 1u << c;
    }
    // the queue order: pipeline distance between the level-2 passes (waits
    // against scratch footprint in L2), the placement of level-1 work, and
    // the tiles or row groups per pass task (hand-over against balance)
    fx::Schedule best = dflt;
    best.variants = vmask;
    float tbest = -1;
    if (fx_rebuild(p, m, n, off, best) == DC_OK) tbest = fx_time(p, s);
    for (int cand : {p->grid / 4, p->grid / 2, p->grid}) {
      for (int mode = 0; mode < fx::kL1Modes; ++mode) {
        for (int units : {1, 2, 4}) {
          fx::Schedule sc{cand, mode, units};
          sc.variants = vmask;
          if (cand < 1 || (cand == dflt.batch_target && mode == dflt.l1_mode && units == dflt.units)) continue;
          if (fx_rebuild(p, m, n, off, sc) != DC_OK) continue;
          const float t = fx_time(p, s);
          if (t > 0 && (tbest < 0 || t < tbest)) { tbest = t; best = sc; }
        }
      }
    }
    cudaStreamDestroy(s);
    cudaGetLastError();
    st = fx_rebuild(p, m, n, off, best);
    if (st != DC_OK) return st;
    p->fx_sched = best;
  }
  return DC_OK;
}
void free_chunks(dc_batched_plan* p) {
  auto& c = p->chunks;
  for (auto* q : c.plans) dc_batched_plan_destroy(q);
  for (auto e : c.ev) cudaEventDestroy(e);
  for (auto& s : c.st)
    if (s) cudaStreamDestroy(s);
  c = dc_batched_plan::Chunks{};
}

// Splits the instances into n chunks of consecutive instances with about
// equal element counts and plans each (same dtype and flags, never the
// one-per-launch mode); streams and events for the pipelined execution.
dc_status make_chunks(dc_batched_plan* p, int n) {
  if (p->chunks.n == n) return DC_OK;
  free_chunks(p);
  auto& c = p->chunks;
  n = std::max(1, std::min(n, p->n));
  // Chunk plans on the fixed-shape engine take the plan's split variants
  // instead of tuning their own: the split changes the rounding, and a
  // host-to-host call gives the device-to-device call's result bit for bit.
  const int flags = p->flags & ~(DC_PLAN_ONE_PER_LAUNCH | (p->fx ? DC_PLAN_AUTOTUNE : 0));
  int32_t i = 0;
  for (int k = 0; k < n && i < p->n; ++k) {
    const int64_t goal = p->total * (k + 1) / n;
    int32_t j = i + 1;
    while (j < p->n && (p->off_host[j] < goal || k == n - 1)) ++j;
    dc_batched_plan* q = nullptr;
    dc_status st = dc_batched_plan_create(p->m_host.data() + i, j - i, p->dtype, flags, &q);
    if (st == DC_OK && p->fx && q->fx && p->inst_first.empty() && p->fx_sched.variants)
      st = dc_batched_plan_set_variants(q, p->fx_sched.variants);
    if (st != DC_OK) {
      if (q) dc_batched_plan_destroy(q);
      free_chunks(p);
      return st;
    }
    c.plans.push_back(q);
    c.first.push_back(i);
    c.work = std::max(c.work, q->work);
    i = j;
  }
  c.first.push_back(p->n);
  for (auto& s : c.st) {
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) { dc_set_last_cuda_error(e); free_chunks(p); return DC_ERR_CUDA; }
  }
  c.ev.resize(3 * c.plans.size() + 5);
  for (auto& e : c.ev) {
    cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (r != cudaSuccess) { dc_set_last_cuda_error(r); free_chunks(p); return DC_ERR_CUDA; }
  }
  c.n = n;
  return DC_OK;
}
}  // namespace

extern "C" {

dc_status dc_batched_plan_create(const int64_t* m, int32_t n, int32_t dtype, int32_t flags,
                                 dc_batched_plan** out) {
  if (!m || n < 1 || !out) return DC_ERR_ARG;
  const int ds = dtype == DC_C64 ? 8 : dtype == DC_C128 ? 16 : 0;
  if (!ds) return DC_ERR_ARG;
  auto* p = new dc_batched_plan();
  p->dtype = dtype; p->ds = ds; p->flags = flags; p->n = n;
  DC_CUDA_TRY(cudaGetDevice(&p->device));
  const int smem_max = device_info().smem_optin - kStaticSmemReserve;
  const bool one = (flags & DC_PLAN_ONE_PER_LAUNCH) != 0;

  std::vector<int64_t> off(n + 1, 0);
  std::map<int64_t, std::vector<int32_t>> by_size;
  for (int32_t i = 0; i < n; ++i) {
    if (m[i] < 1) { delete p; return DC_ERR_ARG; }
    off[i + 1] = off[i] + m[i];
    by_size[m[i]].push_back(i);
  }
  p->total = off[n];
  p->m_host.assign(m, m + n);
  p->off_host = off;

  bool all_fixed = true;
  for (int32_t i = 0; i < n && all_fixed; ++i) all_fixed = fx::f32::size_code(m[i]) >= 0;
  if (all_fixed) {
    dc_status st = create_fixed(p, m, n, off, flags);
    if (st != DC_OK) { delete p; return st; }
    *out = p;
    return DC_OK;
  }

  struct Pending { Item it; double cost; std::vector<int32_t> ids; };
  std::vector<Pending> pend;
  for (auto& kv : by_size) {
    CfgDev c;
    if (!make_cfg(K_COMPLEX, kv.first, ds, kThreads, smem_max, 0, &c)) { delete p; return DC_ERR_SIZE; }
    if ((flags & DC_PLAN_AUTOTUNE) && !one) {
      dc_status st = autotune_size(kv.first, (int)kv.second.size(), ds, smem_max, &c);
      if (st != DC_OK) { delete p; return st; }
    }
    const void* tw = nullptr;
    dc_status st = get_root_table(c.TN, ds, &tw);
    if (st != DC_OK) { delete p; return st; }
    c.tw = tw;
    const int ci = (int)p->cfgs.size();
    p->cfgs.push_back(c);
    p->smem = std::max(p->smem, (int)c.smem);
    p->slot = std::max(p->slot, align_up(cfg_scratch_bytes(K_COMPLEX, c, ds), 256));
    const int per = one ? 1 : (c.level == 1 ? c.nt : 1);
    const auto& ids = kv.second;
    for (size_t s = 0; s < ids.size(); s += per) {
      Pending q;
      q.it.cfg = ci;
      q.it.count = (int32_t)std::min<size_t>(per, ids.size() - s);
      q.ids.assign(ids.begin() + s, ids.begin() + s + q.it.count);
      q.cost = item_cost(c, q.it.count);
      pend.push_back(std::move(q));
    }
  }
  if (one) {
    // the plain mode runs instances in their original order
    std::sort(pend.begin(), pend.end(), [](const Pending& a, const Pending& b) { return a.ids[0] < b.ids[0]; });
  } else {
    std::stable_sort(pend.begin(), pend.end(), [](const Pending& a, const Pending& b) { return a.cost > b.cost; });
  }
  std::vector<int32_t> order;
  for (auto& q : pend) {
    q.it.first = (int32_t)order.size();
    order.insert(order.end(), q.ids.begin(), q.ids.end());
    p->items.push_back(q.it);
  }

  int bps = 1;
  dc_status st = conv1d_blocks_per_sm(K_COMPLEX, ds, p->smem, &bps);
  if (st != DC_OK) { delete p; return st; }
  p->grid = one ? 1 : std::max(1, bps) * device_info().sms;
  p->work = sizeof(WorkHeader) + (size_t)p->grid * p->slot;

  const size_t bc = align_up(p->cfgs.size() * sizeof(CfgDev), 256);
  const size_t bi = align_up(p->items.size() * sizeof(Item), 256);
  const size_t bo = align_up(order.size() * sizeof(int32_t), 256);
  const size_t bf = align_up(off.size() * sizeof(int64_t), 256);
  cudaError_t e = cudaMalloc(&p->dmem, bc + bi + bo + bf);
  if (e != cudaSuccess) { dc_set_last_cuda_error(e); delete p; return DC_ERR_CUDA; }
  p->d_cfgs = (CfgDev*)p->dmem;
  p->d_items = (Item*)(p->dmem + bc);
  p->d_order = (int32_t*)(p->dmem + bc + bi);
  p->d_off = (int64_t*)(p->dmem + bc + bi + bo);
  e = cudaMemcpy(p->d_cfgs, p->cfgs.data(), p->cfgs.size() * sizeof(CfgDev), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_items, p->items.data(), p->items.size() * sizeof(Item), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_order, order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { dc_set_last_cuda_error(e); cudaFree(p->dmem); delete p; return DC_ERR_CUDA; }
  *out = p;
  return DC_OK;
}

dc_status dc_batched_plan_workspace_size(const dc_batched_plan* p, size_t* bytes) {
  if (!p || !bytes) return DC_ERR_ARG;
  *bytes = p->work;
  return DC_OK;
}

dc_status dc_batched_plan_launches(const dc_batched_plan* p, int32_t* launches) {
  if (!p || !launches) return DC_ERR_ARG;
  if (p->fx) *launches = p->inst_first.empty() ? 1 : (int32_t)p->inst_first.size();
  else *launches = (p->flags & DC_PLAN_ONE_PER_LAUNCH) ? (int32_t)p->items.size() : 1;
  return DC_OK;
}

dc_status dc_selftest_wait_timeout(void* work, size_t work_bytes, int64_t cycles, void* stream) {
  // header | one counter (never advanced) | one task waiting for it
  const size_t need = 256 + 256 + sizeof(fx::Task);
  if (!work || cycles < 1) return DC_ERR_ARG;
  if ((uintptr_t)work % 256) return DC_ERR_ALIGN;
  if (work_bytes < need) return DC_ERR_NOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  int bps = 0;
  dc_status st = fx::f32::prepare_kernel(fx_smem_all(&kFx32), &bps);
  if (st != DC_OK) return st;
  static const fx::Task task{(fx::T_B << 8) | 0, 0, 0, 0, 1u, -1};
  char* w = (char*)work;
  DC_CUDA_TRY(cudaMemsetAsync(w, 0, 512, s));
  DC_CUDA_TRY(cudaMemcpyAsync(w + 512, &task, sizeof(task), cudaMemcpyHostToDevice, s));
  fx::FxArgs a{};
  a.tasks = (const fx::Task*)(w + 512);
  a.ntasks = 1;
  a.hdr = (WorkHeader*)w;
  a.cnt = (uint32_t*)(w + 256);
  a.wait_limit = cycles;
  // one block: it takes the task, waits, records the timeout and leaves
  return fx::f32::launch(a, 1, fx::f32::code_smem(0), s);
}

dc_status dc_batched_plan_schedule(const dc_batched_plan* p, int32_t* batch_target, int32_t* l1_mode) {
  if (!p || !p->fx || !p->inst_first.empty()) return DC_ERR_ARG;
  if (batch_target) *batch_target = p->fx_sched.batch_target;
  if (l1_mode) *l1_mode = p->fx_sched.l1_mode;
  return DC_OK;
}

dc_status dc_batched_plan_set_schedule(dc_batched_plan* p, int32_t batch_target, int32_t l1_mode) {
  if (!p || !p->fx || !p->inst_first.empty() || batch_target < 1 || l1_mode < 0 || l1_mode >= fx::kL1Modes)
    return DC_ERR_ARG;
  std::vector<int64_t> ms(p->n);
  for (int32_t i = 0; i < p->n; ++i) ms[i] = p->off_host[i + 1] - p->off_host[i];
  fx::Schedule sc{batch_target, l1_mode, p->fx_sched.units};
  sc.variants = p->fx_sched.variants;
  dc_status st = fx_rebuild(p, ms.data(), p->n, p->off_host, sc);
  if (st != DC_OK) return st;
  p->fx_sched = sc;
  return DC_OK;
}

dc_status dc_batched_plan_task_units(const dc_batched_plan* p, int32_t* units) {
  if (!p || !p->fx || !p->inst_first.empty() || !units) return DC_ERR_ARG;
  *units = p->fx_sched.units;
  return DC_OK;
}

dc_status dc_batched_plan_set_task_units(dc_batched_plan* p, int32_t units) {
  if (!p || !p->fx || !p->inst_first.empty() || units < 1 || units > fx::kMaxUnits) return DC_ERR_ARG;
  std::vector<int64_t> ms(p->n);
  for (int32_t i = 0; i < p->n; ++i) ms[i] = p->off_host[i + 1] - p->off_host[i];
  fx::Schedule sc{p->fx_sched.batch_target, p->fx_sched.l1_mode, units};
  sc.variants = p->fx_sched.variants;
  dc_status st = fx_rebuild(p, ms.data(), p->n, p->off_host, sc);
  if (st != DC_OK) return st;
  p->fx_sched = sc;
  return DC_OK;
}

dc_status dc_batched_plan_variants(const dc_batched_plan* p, uint32_t* mask) {
  if (!p || !p->fx || !p->inst_first.empty() || !mask) return DC_ERR_ARG;
  *mask = p->fx_sched.variants;
  return DC_OK;
}

dc_status dc_batched_plan_set_variants(dc_batched_plan* p, uint32_t mask) {
  if (!p || !p->fx || !p->inst_first.empty()) return DC_ERR_ARG;
  std::vector<int64_t> ms(p->n);
  for (int32_t i = 0; i < p->n; ++i) ms[i] = p->off_host[i + 1] - p->off_host[i];
  fx::Schedule sc = p->fx_sched;
  // only sizes that have a second split keep their bit
  sc.variants = 0;
  for (int c = 0; c < fx::kNumSizes; ++c)
    if (((mask >> c) & 1u) && p->ops->code_ok(c + fx::kCodeStride, p->mode)) sc.variants |= 1u << c;
  dc_status st = fx_rebuild(p, ms.data(), p->n, p->off_host, sc);
  if (st != DC_OK) return st;
  p->fx_sched = sc;
  free_chunks(p);   // the host pipeline's chunk plans follow the new variants
  return DC_OK;
}

dc_status dc_batched_plan_describe(const dc_batched_plan* p, int32_t i, int64_t* m, int32_t* level,
                                   int32_t* nt, int32_t* l1, int32_t* l2, int32_t* w) {
  if (p && p->fx) {
    if (i < 0 || i >= (int32_t)p->hp.codes.size()) return DC_ERR_ARG;
    int lv, per, a, b, ww;
    p->ops->code_shape(p->hp.codes[i], &lv, &per, &a, &b, &ww);
    if (m) *m = p->ops->code_size(p->hp.codes[i]);
    if (level) *level = lv;
    if (nt) *nt = per;
    if (l1) *l1 = a;
    if (l2) *l2 = b;
    if (w) *w = ww;
    return DC_OK;
  }
  if (!p || i < 0 || i >= (int32_t)p->cfgs.size()) return DC_ERR_ARG;
  const CfgDev& c = p->cfgs[i];
  if (m) *m = c.m;
  if (level) *level = c.level;
  if (nt) *nt = c.nt;
  if (l1) *l1 = c.L1;
  if (l2) *l2 = c.L2;
  if (w) *w = c.w;
  return DC_OK;
}

dc_status dc_conv_complex_1d_batched(const dc_batched_plan* p, const void* f, const void* g,
                                     void* h, void* work, size_t work_bytes, void* stream) {
  if (!p || !f || !g || !h || !work) return DC_ERR_ARG;
  const size_t a8 = (size_t)p->ds;
  if ((uintptr_t)f % a8 || (uintptr_t)g % a8 || (uintptr_t)h % a8 || (uintptr_t)work % 256)
    return DC_ERR_ALIGN;
  if (work_bytes < p->work) return DC_ERR_NOMEM;
  const size_t bytes = (size_t)p->total * p->ds;
  auto overl = [bytes](const void* o, const void* i) {
    if (o == i) return false;
    const char* a = (const char*)o;
    const char* b = (const char*)i;
    return a < b + bytes && b < a + bytes;
  };
  if (overl(h, f) || overl(h, g)) return DC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (p->fx) return fx_launch(p, f, g, h, work, s);
  ConvArgs a{};
  a.in[0] = f;
  a.in[1] = g;
  a.out[0] = h;
  a.off = p->d_off;
  a.order = p->d_order;
  a.cfgs = p->d_cfgs;
  a.hdr = (WorkHeader*)work;
  a.scratch = (char*)work + sizeof(WorkHeader);
  a.slot_bytes = (int64_t)p->slot;
  a.ninst = p->n;
  DC_CUDA_TRY(cudaMemsetAsync(work, 0, sizeof(WorkHeader), s));
  if (p->flags & DC_PLAN_ONE_PER_LAUNCH) {
    for (size_t j = 0; j < p->items.size(); ++j) {
      a.items = p->d_items + j;
      a.nitems = 1;
      a.persistent = 0;
      dc_status st = launch_conv1d(K_COMPLEX, p->ds, a, 1, p->cfgs[p->items[j].cfg].smem, s);
      if (st != DC_OK) return st;
    }
    return DC_OK;
  }
  a.items = p->d_items;
  a.nitems = (int32_t)p->items.size();
  a.persistent = 1;
  return launch_conv1d(K_COMPLEX, p->ds, a, p->grid, p->smem, s);
}

dc_status dc_batched_plan_host_workspace_size(dc_batched_plan* p, int32_t nchunks, size_t* bytes) {
  if (!p || !bytes || nchunks < 1) return DC_ERR_ARG;
  dc_status st = make_chunks(p, nchunks);
  if (st != DC_OK) return st;
  *bytes = p->chunks.work;
  return DC_OK;
}

dc_status dc_conv_complex_1d_batched_host(dc_batched_plan* p, const void* hf, const void* hg, void* hh,
                                          void* df, void* dg, void* dh, void* work, size_t work_bytes,
                                          int32_t nchunks, void* stream) {
  if (!p || !hf || !hg || !hh || !df || !dg || !dh || !work || nchunks < 1) return DC_ERR_ARG;
  const size_t a8 = (size_t)p->ds;
  if ((uintptr_t)df % a8 || (uintptr_t)dg % a8 || (uintptr_t)dh % a8 || (uintptr_t)work % 256)
    return DC_ERR_ALIGN;
  dc_status st = make_chunks(p, nchunks);
  if (st != DC_OK) return st;
  auto& c = p->chunks;
  if (work_bytes < c.work) return DC_ERR_NOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  const int nc = (int)c.plans.size();
  cudaEvent_t* evf = &c.ev[0];
  cudaEvent_t* evh = &c.ev[nc];
  cudaEvent_t* evg = &c.ev[2 * nc];
  cudaEvent_t start = c.ev[3 * nc], j0 = c.ev[3 * nc + 1], j1 = c.ev[3 * nc + 2], j2 = c.ev[3 * nc + 3],
              j3 = c.ev[3 * nc + 4];
  // the four streams start after the work already on `stream`
  DC_CUDA_TRY(cudaEventRecord(start, s));
  for (auto& q : c.st) DC_CUDA_TRY(cudaStreamWaitEvent(q, start, 0));
  auto bytes_of = [&](int k) { return (size_t)(p->off_host[c.first[k + 1]] - p->off_host[c.first[k]]) * a8; };
  auto at = [&](const void* base, int k) { return (const char*)base + (size_t)p->off_host[c.first[k]] * a8; };
  // Everything from here on is enqueued on the forked streams; whatever
  // fails, `stream` is joined to them before returning, so that copies
  // already queued on the caller's host buffers finish before any later
  // work on `stream` (or a synchronize of it) lets the caller reuse them.
  auto enqueue = [&]() -> dc_status {
    // f and g come in on one stream (a second one measured no faster: the
    // host link is the limit), h goes out on another
    for (int k = 0; k < nc; ++k) {
      DC_CUDA_TRY(cudaMemcpyAsync((void*)at(df, k), at(hf, k), bytes_of(k), cudaMemcpyHostToDevice, c.st[0]));
      DC_CUDA_TRY(cudaEventRecord(evf[k], c.st[0]));
      DC_CUDA_TRY(cudaMemcpyAsync((void*)at(dg, k), at(hg, k), bytes_of(k), cudaMemcpyHostToDevice, c.st[0]));
      DC_CUDA_TRY(cudaEventRecord(evg[k], c.st[0]));
    }
    for (int k = 0; k < nc; ++k) {
      DC_CUDA_TRY(cudaStreamWaitEvent(c.st[1], evf[k], 0));
      DC_CUDA_TRY(cudaStreamWaitEvent(c.st[1], evg[k], 0));
      const dc_status e = dc_conv_complex_1d_batched(c.plans[k], at(df, k), at(dg, k), (void*)at(dh, k), work,
                                                     work_bytes, c.st[1]);
      if (e != DC_OK) return e;
      DC_CUDA_TRY(cudaEventRecord(evh[k], c.st[1]));
    }
    for (int k = 0; k < nc; ++k) {
      DC_CUDA_TRY(cudaStreamWaitEvent(c.st[2], evh[k], 0));
      DC_CUDA_TRY(cudaMemcpyAsync((void*)at(hh, k), at(dh, k), bytes_of(k), cudaMemcpyDeviceToHost, c.st[2]));
    }
    return DC_OK;
  };
  st = enqueue();
  // `stream` continues after all four, on success and on failure alike
  const cudaEvent_t joins[4] = {j0, j1, j2, j3};
  for (int q = 0; q < 4; ++q) {
    const cudaError_t e1 = cudaEventRecord(joins[q], c.st[q]);
    const cudaError_t e2 = e1 == cudaSuccess ? cudaStreamWaitEvent(s, joins[q], 0) : e1;
    if (e2 != cudaSuccess && st == DC_OK) {
      dc_set_last_cuda_error(e2);
      st = DC_ERR_CUDA;
    }
  }
  return st;
}

dc_status dc_batched_plan_destroy(dc_batched_plan* p) {
  if (!p) return DC_ERR_ARG;
  free_chunks(p);
  if (p->dmem) cudaFree(p->dmem);
  delete p;
  return DC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Uniform batches on the fixed-shape engine: n instances of size m at stride
// m (the single 1D complex call, the row convolutions of the multi-D complex
// paths).  Plans are created on first use per (device, n, m, precision) and
// kept until exit, like the root tables.
// ---------------------------------------------------------------------------
#include <mutex>
#include <tuple>

namespace dc {
namespace {
std::mutex g_umu;
std::map<std::tuple<int, int64_t, int64_t, int, int>, dc_batched_plan*> g_uplans;
}  // namespace

bool fx_uniform_ok(int64_t m, int ds) { return (ds == 8 || ds == 16) && fx::f32::size_code(m) >= 0; }

bool fx_uniform_two_level(int64_t m) {
  const int c = fx::f32::size_code(m);
  if (c < 0) return false;
  int lv, per, l1, l2, w;
  fx::f32::code_shape(c, &lv, &per, &l1, &l2, &w);   // the same split in both precisions
  return lv == 2;
}

namespace {
std::map<std::tuple<int, int64_t, int64_t, int, int>, size_t> g_uwork;   // (device, n, m, ds, mode) -> bytes
}  // namespace

size_t fx_uniform_work_uncached(int64_t n, int64_t m, int ds, int mode);

// cached: the query runs on every multi-D and 1D call
size_t fx_uniform_work(int64_t n, int64_t m, int ds, int mode) {
  const auto key = std::make_tuple(device_info().device, n, m, ds, mode);
  {
    std::lock_guard<std::mutex> lock(g_umu);
    auto it = g_uwork.find(key);
    if (it != g_uwork.end()) return it->second;
  }
  const size_t b = fx_uniform_work_uncached(n, m, ds, mode);
  std::lock_guard<std::mutex> lock(g_umu);
  g_uwork[key] = b;
  return b;
}

size_t fx_uniform_work_uncached(int64_t n, int64_t m, int ds, int mode) {
  const FxOps* ops = ds == 8 ? &kFx32 : &kFx64;
  const int bps = ds == 8 ? 2 : 1;   // the kernel's blocks per SM (launch bounds)
  std::vector<int64_t> ms((size_t)n, m), off((size_t)n + 1, 0);
  for (int64_t i = 0; i < n; ++i) off[i + 1] = off[i] + m;
  fx::HostPlan hp;
  const fx::Schedule sc{bps * device_info().sms / 2, 0};
  if (!ops->build_plan(ms.data(), (int32_t)n, off.data(), sc, mode, &hp)) return 0;
  return align_up(sizeof(WorkHeader) + hp.ncnt * sizeof(uint32_t), 256) + align_up(hp.scratch * (size_t)ds, 256) +
         hp.l1_elems * (size_t)ds;
}

dc_status fx_uniform_plan(int64_t n, int64_t m, int ds, dc_batched_plan** out, int mode) {
  int dev = 0;
  DC_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_umu);
  auto key = std::make_tuple(dev, n, m, ds, mode);
  auto it = g_uplans.find(key);
  if (it != g_uplans.end()) { *out = it->second; return DC_OK; }
  std::vector<int64_t> ms((size_t)n, m);
  dc_batched_plan* p = nullptr;
  if (mode == fx::MODE_COMPLEX) {
    dc_status st = dc_batched_plan_create(ms.data(), (int32_t)n, ds == 8 ? DC_C64 : DC_C128, 0, &p);
    if (st != DC_OK) return st;
  } else {
    p = new dc_batched_plan();
    p->dtype = ds == 8 ? DC_C64 : DC_C128;
    p->ds = ds;
    p->n = (int32_t)n;
    std::vector<int64_t> off((size_t)n + 1, 0);
    for (int64_t i = 0; i < n; ++i) off[i + 1] = off[i] + m;
    p->total = off[n];
    p->m_host = ms;
    p->off_host = off;
    DC_CUDA_TRY(cudaGetDevice(&p->device));
    dc_status st = create_fixed(p, ms.data(), (int32_t)n, off, 0, mode);
    if (st != DC_OK) { dc_batched_plan_destroy(p); return st; }
  }
  g_uplans[key] = p;
  *out = p;
  return DC_OK;
}

namespace {
std::map<std::tuple<int, int64_t, int64_t, int>, dc_batched_plan*> g_tplans;   // (device, n, m, ds)
}  // namespace

bool fx_ternary_ok(int64_t m, int ds) { return fx_uniform_ok(2 * m, ds) && fx_uniform_two_level(2 * m); }

size_t fx_ternary_work(int64_t m, int ds, int64_t n) { return fx_uniform_work(n, 2 * m, ds, fx::MODE_TERN); }

// The plan of n ternary convolutions of length m at stride m on the fixed
// engine (n instances of the M = 2m point sub-transforms whose inputs and
// outputs hold m elements: one 1D call, or the rows of a multi-D call),
// cached per device, count and precision.
dc_status fx_ternary_plan(int64_t m, int ds, dc_batched_plan** out, int64_t n) {
  if (!fx_ternary_ok(m, ds) || n < 1) return DC_ERR_SIZE;
  int dev = 0;
  DC_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_umu);
  auto key = std::make_tuple(dev, n, m, ds);
  auto it = g_tplans.find(key);
  if (it != g_tplans.end()) { *out = it->second; return DC_OK; }
  std::vector<int64_t> ms((size_t)n, 2 * m), off((size_t)n + 1, 0);
  for (int64_t i = 0; i < n; ++i) off[i + 1] = off[i] + m;
  dc_batched_plan* p = new dc_batched_plan();
  p->dtype = ds == 8 ? DC_C64 : DC_C128;
  p->ds = ds;
  p->n = (int32_t)n;
  p->total = n * m;
  p->m_host = ms;
  p->off_host = off;
  p->device = dev;
  dc_status st = create_fixed(p, ms.data(), (int32_t)n, off, 0, fx::MODE_TERN);
  if (st != DC_OK) { dc_batched_plan_destroy(p); return st; }
  g_tplans[key] = p;
  *out = p;
  return DC_OK;
}

dc_status fx_ternary_run(int64_t m, int ds, const void* f, const void* g, const void* e, void* h, void* work,
                         size_t work_bytes, cudaStream_t s, int64_t n) {
  dc_batched_plan* p = nullptr;
  dc_status st = fx_ternary_plan(m, ds, &p, n);
  if (st != DC_OK) return st;
  if (work_bytes < p->work) return DC_ERR_NOMEM;
  return fx_launch(p, f, g, h, work, s, e);
}

dc_status fx_hdot2_run(dc_batched_plan* p, const void* f1, const void* g1, const void* f2, const void* g2, void* h,
                       void* work, size_t work_bytes, cudaStream_t s) {
  if (!p || p->mode != fx::MODE_HDOT2) return DC_ERR_ARG;
  if (work_bytes < p->work) return DC_ERR_NOMEM;
  return fx_launch(p, f1, g1, h, work, s, f2, nullptr, g2);
}

dc_status fx_tern4_run(dc_batched_plan* p, const void* f, const void* g, const void* e, void* h, void* work,
                       size_t work_bytes, cudaStream_t s) {
  if (!p || p->mode != fx::MODE_TERN4) return DC_ERR_ARG;
  if (work_bytes < p->work) return DC_ERR_NOMEM;
  return fx_launch(p, f, g, h, work, s, e);
}

dc_status fx_pair_run(dc_batched_plan* p, const void* w, const void* f, const void* g, void* df, void* dg,
                      void* work, size_t work_bytes, cudaStream_t s) {
  if (!p || p->mode != fx::MODE_PAIR) return DC_ERR_ARG;
  if (work_bytes < p->work) return DC_ERR_NOMEM;
  return fx_launch(p, w, f, df, work, s, g, dg);
}

}  // namespace dc

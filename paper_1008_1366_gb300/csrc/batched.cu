// Batched 1D complex convolutions of uneven sizes in one persistent launch.
//
// Planning groups the instances by size; each size gets a configuration
// (level 1: `nt` instances per block wholly in shared memory; level 2: one
// instance per block through a scratch slot).  Work items (a group of same-
// size instances, or one large instance) are sorted by estimated cost,
// largest first, and a persistent grid of (SMs x resident blocks) takes them
// from an atomic counter, which balances uneven sizes like a longest-
// processing-time schedule.
#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

#include "conv1d.cuh"
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
};

namespace {
size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

double item_cost(const CfgDev& c, int count) {
  // six sub-transforms of length L per instance plus the level-2 passes
  double f = 6.0 * (double)std::max<int64_t>(fft_flops(c.L), c.L) * count;
  if (c.level == 2) f *= 1.5;
  return f;
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

  struct Pending { Item it; double cost; std::vector<int32_t> ids; };
  std::vector<Pending> pend;
  for (auto& kv : by_size) {
    CfgDev c;
    if (!make_cfg(K_COMPLEX, kv.first, ds, kThreads, smem_max, 0, &c)) { delete p; return DC_ERR_SIZE; }
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
  *launches = (p->flags & DC_PLAN_ONE_PER_LAUNCH) ? (int32_t)p->items.size() : 1;
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

dc_status dc_batched_plan_destroy(dc_batched_plan* p) {
  if (!p) return DC_ERR_ARG;
  if (p->dmem) cudaFree(p->dmem);
  delete p;
  return DC_OK;
}

}  // extern "C"

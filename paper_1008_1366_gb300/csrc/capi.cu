// C ABI entry points (include/dealias.h): argument checks, planning and
// dispatch to the kernels.  No entry point allocates device memory except
// the first use of a size (root tables) and plan creation.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "conv1d.cuh"
#include "fixed.h"
#include "launch.h"
#include "multid.h"
#include "plan.h"
#include "tables.h"

using namespace dc;

namespace {
thread_local int32_t t_last_cuda = 0;
std::mutex g_dev_mu;
DeviceInfo g_dev[64];
bool g_dev_ok[64] = {false};
}  // namespace

extern "C" void dc_set_last_cuda_error(cudaError_t e) { t_last_cuda = (int32_t)e; }

namespace dc {
const DeviceInfo& device_info() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  std::lock_guard<std::mutex> lock(g_dev_mu);
  if (!g_dev_ok[dev]) {
    DeviceInfo d{};
    d.device = dev;
    cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&d.l2_bytes, cudaDevAttrL2CacheSize, dev);
    if (d.sms <= 0) d.sms = 1;
    if (d.smem_optin <= 0) d.smem_optin = 48 * 1024;
    g_dev[dev] = d;
    g_dev_ok[dev] = true;
  }
  return g_dev[dev];
}
}  // namespace dc

namespace {

constexpr size_t kHeader = sizeof(WorkHeader);

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int dsize_of(int32_t dtype) { return dtype == DC_C64 ? 8 : dtype == DC_C128 ? 16 : 0; }

int smem_budget() { return device_info().smem_optin - kStaticSmemReserve; }

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// Output may equal an input exactly; partial overlap is an error.
bool bad_overlap(const void* o, const void* i, size_t bytes) {
  if (!o || !i || o == i) return false;
  const char* a = (const char*)o;
  const char* b = (const char*)i;
  return a < b + bytes && b < a + bytes;
}

dc_status check_ptrs(const void* const* ins, int nin, void* const* outs, int nout, size_t bytes,
                     int ds) {
  for (int x = 0; x < nin; ++x) {
    if (!ins[x]) return DC_ERR_ARG;
    if (!aligned(ins[x], ds)) return DC_ERR_ALIGN;
  }
  for (int o = 0; o < nout; ++o) {
    if (!outs[o]) return DC_ERR_ARG;
    if (!aligned(outs[o], ds)) return DC_ERR_ALIGN;
    for (int x = 0; x < nin; ++x)
      if (bad_overlap(outs[o], ins[x], bytes)) return DC_ERR_ARG;
    for (int p = 0; p < o; ++p)
      if (outs[p] == outs[o] || bad_overlap(outs[o], outs[p], bytes)) return DC_ERR_ARG;
  }
  return DC_OK;
}

dc_status check_work(void* work, size_t have, size_t need) {
  if (!work) return DC_ERR_ARG;
  if (!aligned(work, 256)) return DC_ERR_ALIGN;
  if (have < need) return DC_ERR_NOMEM;
  return DC_OK;
}

int fixed_mode(int kind) { return kind == K_HERMITIAN ? fx::MODE_HERM : fx::MODE_COMPLEX; }

bool on_fixed_engine(int kind, int64_t m, int ds) {
  return (kind == K_COMPLEX || kind == K_HERMITIAN) && fx_uniform_ok(m, ds) && fx_uniform_two_level(m);
}

// Plans one 1D call; fills cfg (with its table) and the workspace size.
dc_status plan_1d(int kind, int64_t m, int ds, bool with_table, CfgDev* cfg, size_t* work) {
  if (m < 1) return DC_ERR_ARG;
  if (!make_cfg(kind, m, ds, kThreads, smem_budget(), 0, cfg)) return DC_ERR_SIZE;
  if (with_table) {
    const void* tw = nullptr;
    dc_status st = get_root_table(cfg->TN, ds, &tw);
    if (st != DC_OK) return st;
    cfg->tw = tw;
  }
  *work = kHeader + align_up(cfg_scratch_bytes(kind, *cfg, ds), 256);
  // a single binary complex or centered Hermitian convolution of a
  // two-level size runs on the fixed-shape engine (a one-instance plan,
  // cached): its passes spread over many blocks, where the runtime-shaped
  // kernel gives the instance one
  if (on_fixed_engine(kind, m, ds)) {
    *work = std::max(*work, fx_uniform_work(1, m, ds, fixed_mode(kind)));
    if (with_table) {
      dc_batched_plan* p = nullptr;
      dc_status st = fx_uniform_plan(1, m, ds, &p, fixed_mode(kind));
      if (st != DC_OK) return st;
    }
  }
  // likewise a ternary convolution whose 2m-point sub-transforms are a
  // two-level size
  if (kind == K_TERNARY && fx_ternary_ok(m, ds)) {
    *work = std::max(*work, fx_ternary_work(m, ds));
    if (with_table) {
      dc_batched_plan* p = nullptr;
      dc_status st = fx_ternary_plan(m, ds, &p);
      if (st != DC_OK) return st;
    }
  }
  return DC_OK;
}

dc_status run_1d(int kind, const void* const* ins, int nin, void* const* outs, int nout, int64_t m,
                 int32_t dtype, void* work, size_t work_bytes, void* stream) {
  const int ds = dsize_of(dtype);
  if (!ds || m < 1) return DC_ERR_ARG;
  dc_status st = check_ptrs(ins, nin, outs, nout, (size_t)m * ds, ds);
  if (st != DC_OK) return st;
  CfgDev cfg;
  size_t need = 0;
  st = plan_1d(kind, m, ds, true, &cfg, &need);
  if (st != DC_OK) return st;
  if ((st = check_work(work, work_bytes, need)) != DC_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (on_fixed_engine(kind, m, ds)) {
    dc_batched_plan* p = nullptr;
    if ((st = fx_uniform_plan(1, m, ds, &p, fixed_mode(kind))) != DC_OK) return st;
    return dc_conv_complex_1d_batched(p, ins[0], ins[1], outs[0], work, work_bytes, s);
  }
  if (kind == K_TERNARY && fx_ternary_ok(m, ds))
    return fx_ternary_run(m, ds, ins[0], ins[1], ins[2], outs[0], work, work_bytes, s);
  ConvArgs a{};
  for (int x = 0; x < nin; ++x) a.in[x] = ins[x];
  for (int o = 0; o < nout; ++o) a.out[o] = outs[o];
  a.nitems = 1;
  a.ninst = 1;
  a.hdr = (WorkHeader*)work;
  a.scratch = (char*)work + kHeader;
  a.slot_bytes = (int64_t)align_up(cfg_scratch_bytes(kind, cfg, ds), 256);
  a.cfg0 = cfg;
  DC_CUDA_TRY(cudaMemsetAsync(work, 0, kHeader, s));
  return launch_conv1d(kind, ds, a, 1, cfg.smem, s);
}

dc_status run_md(int32_t pk, int ndim, const int64_t* dims, const void* const* ins, int nin,
                 void* const* outs, int nout, int32_t dtype, void* work, size_t work_bytes,
                 void* stream) {
  const int ds = dsize_of(dtype);
  if (!ds) return DC_ERR_ARG;
  for (int d = 0; d < ndim; ++d) if (dims[d] < 1) return DC_ERR_ARG;
  const bool herm = pk == DC_KIND_HERMITIAN || pk == DC_KIND_HERMITIAN_ADJOINT || pk == DC_KIND_HERMITIAN_DOT2 ||
                    pk == DC_KIND_TERNARY;
  int64_t n = 1;
  for (int d = 0; d < ndim; ++d) n *= (herm && d < ndim - 1) ? 2 * dims[d] - 1 : dims[d];
  dc_status st = check_ptrs(ins, nin, outs, nout, (size_t)n * ds, ds);
  if (st != DC_OK) return st;
  if (!work) return DC_ERR_ARG;
  if (!aligned(work, 256)) return DC_ERR_ALIGN;
  return md_run(pk, ndim, dims, ds, ins, nin, outs, nout, work, work_bytes, (cudaStream_t)stream);
}

int kind_of_public(int32_t k) {
  switch (k) {
    case DC_KIND_COMPLEX: return K_COMPLEX;
    case DC_KIND_HERMITIAN: return K_HERMITIAN;
    case DC_KIND_TERNARY: return K_TERNARY;
    case DC_KIND_COMPLEX_ADJOINT: return K_COMPLEX_ADJ;
    case DC_KIND_HERMITIAN_ADJOINT: return K_HERMITIAN_ADJ;
    case DC_KIND_COMPLEX_DOT2: return K_COMPLEX_DOT2;
    case DC_KIND_HERMITIAN_DOT2: return K_HERMITIAN_DOT2;
  }
  return -1;
}

}  // namespace

extern "C" {

const char* dc_status_string(dc_status s) {
  switch (s) {
    case DC_OK: return "ok";
    case DC_ERR_ARG: return "invalid argument";
    case DC_ERR_SIZE: return "unsupported size";
    case DC_ERR_ALIGN: return "misaligned pointer";
    case DC_ERR_CUDA: return "CUDA runtime error";
    case DC_ERR_TIMEOUT: return "device-side wait timed out";
    case DC_ERR_NOMEM: return "workspace too small";
    case DC_ERR_DEVICE: return "device-side check failed";
  }
  return "unknown status";
}

int32_t dc_last_cuda_error(void) { return t_last_cuda; }

dc_status dc_workspace_size(int32_t kind, int32_t ndim, const int64_t* dims, int32_t dtype,
                            size_t* bytes) {
  const int ds = dsize_of(dtype);
  const int k = kind_of_public(kind);
  if (!ds || k < 0 || !dims || !bytes || ndim < 1 || ndim > 3) return DC_ERR_ARG;
  if (ndim > 1) return md_workspace(kind, ndim, dims, ds, bytes);
  CfgDev cfg;
  return plan_1d(k, dims[0], ds, false, &cfg, bytes);
}

dc_status dc_workspace_size_slabs(int32_t kind, int32_t ndim, const int64_t* dims, int32_t dtype,
                                  int64_t slabs_per_chunk, size_t* bytes) {
  const int ds = dsize_of(dtype);
  const int k = kind_of_public(kind);
  if (!ds || k < 0 || !dims || !bytes || ndim != 3 || slabs_per_chunk < 1) return DC_ERR_ARG;
  return md_workspace_slabs(kind, ndim, dims, ds, slabs_per_chunk, bytes);
}

dc_status dc_chunking(int32_t kind, int32_t ndim, const int64_t* dims, int32_t dtype, size_t work_bytes,
                      int64_t* slabs_per_chunk, int64_t* chunks) {
  const int ds = dsize_of(dtype);
  const int k = kind_of_public(kind);
  if (!ds || k < 0 || !dims || !slabs_per_chunk || !chunks || ndim < 2 || ndim > 3) return DC_ERR_ARG;
  return md_chunking(kind, ndim, dims, ds, work_bytes, slabs_per_chunk, chunks);
}

dc_status dc_prepare(int32_t kind, int32_t ndim, const int64_t* dims, int32_t dtype) {
  const int ds = dsize_of(dtype);
  const int k = kind_of_public(kind);
  if (!ds || k < 0 || !dims || ndim < 1 || ndim > 3) return DC_ERR_ARG;
  if (ndim > 1) return md_prepare(kind, ndim, dims, ds);
  CfgDev cfg;
  size_t need;
  return plan_1d(k, dims[0], ds, true, &cfg, &need);
}

dc_status dc_read_status(const void* work, void* stream, int32_t* status, int32_t* detail) {
  if (!work || !status) return DC_ERR_ARG;
  WorkHeader h;
  DC_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  DC_CUDA_TRY(cudaMemcpy(&h, work, sizeof(h), cudaMemcpyDeviceToHost));
  *status = h.status;
  if (detail) *detail = h.detail;
  return DC_OK;
}

dc_status dc_read_trace(const void* work, void* stream, uint64_t* out) {
  if (!work || !out) return DC_ERR_ARG;
  WorkHeader h;
  DC_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  DC_CUDA_TRY(cudaMemcpy(&h, work, sizeof(h), cudaMemcpyDeviceToHost));
  out[0] = h.waited;
  out[1] = h.wait_cycles;
  for (int k = 0; k < 4; ++k) {
    out[2 + k] = h.type_cycles[k];
    out[6 + k] = h.type_count[k];
  }
  out[10] = h.handover_cycles;
  out[11] = h.table_cycles;
  return DC_OK;
}

dc_status dc_conv_complex_1d(const void* f, const void* g, void* h, int64_t m, int32_t dtype,
                             void* work, size_t work_bytes, void* stream) {
  const void* ins[2] = {f, g};
  void* outs[1] = {h};
  return run_1d(K_COMPLEX, ins, 2, outs, 1, m, dtype, work, work_bytes, stream);
}

dc_status dc_conv_hermitian_1d(const void* f, const void* g, void* h, int64_t m, int32_t dtype,
                               void* work, size_t work_bytes, void* stream) {
  const void* ins[2] = {f, g};
  void* outs[1] = {h};
  return run_1d(K_HERMITIAN, ins, 2, outs, 1, m, dtype, work, work_bytes, stream);
}

dc_status dc_conv_ternary_hermitian_1d(const void* f, const void* g, const void* e, void* h,
                                       int64_t m, int32_t dtype, void* work, size_t work_bytes,
                                       void* stream) {
  const void* ins[3] = {f, g, e};
  void* outs[1] = {h};
  return run_1d(K_TERNARY, ins, 3, outs, 1, m, dtype, work, work_bytes, stream);
}

dc_status dc_conv_complex_1d_adjoint(const void* w, const void* f, const void* g, void* df,
                                     void* dg, int64_t m, int32_t dtype, void* work,
                                     size_t work_bytes, void* stream) {
  const void* ins[3] = {w, f, g};
  void* outs[2] = {df, dg};
  return run_1d(K_COMPLEX_ADJ, ins, 3, outs, 2, m, dtype, work, work_bytes, stream);
}

dc_status dc_conv_hermitian_1d_adjoint(const void* w, const void* f, const void* g, void* df,
                                       void* dg, int64_t m, int32_t dtype, void* work,
                                       size_t work_bytes, void* stream) {
  const void* ins[3] = {w, f, g};
  void* outs[2] = {df, dg};
  return run_1d(K_HERMITIAN_ADJ, ins, 3, outs, 2, m, dtype, work, work_bytes, stream);
}

dc_status dc_workspace_size_pq(int64_t m, int32_t p, int32_t q, int64_t nout, int32_t dtype, size_t* bytes) {
  const int ds = dsize_of(dtype);
  if (!ds || !bytes) return DC_ERR_ARG;
  FftPlan plan;
  return pq_plan(m, p, q, nout, ds, &plan, bytes);
}

dc_status dc_conv_complex_1d_pq(const void* f, const void* g, void* h, int64_t m, int32_t p, int32_t q,
                                int64_t nout, int32_t dtype, void* work, size_t work_bytes, void* stream) {
  const int ds = dsize_of(dtype);
  if (!ds || m < 1 || p < 1 || nout < 1) return DC_ERR_ARG;
  // inputs hold p m values, the output nout; h may be f or g, no other overlap
  if (!f || !g || !h) return DC_ERR_ARG;
  if (!aligned(f, ds) || !aligned(g, ds) || !aligned(h, ds)) return DC_ERR_ALIGN;
  const size_t in_bytes = (size_t)p * m * ds, out_bytes = (size_t)nout * ds;
  for (const void* x : {f, g}) {
    const char* a = (const char*)h;
    const char* b = (const char*)x;
    if (x != h && a < b + in_bytes && b < a + out_bytes) return DC_ERR_ARG;
  }
  dc_status st = DC_OK;
  FftPlan plan;
  size_t need = 0;
  if ((st = pq_plan(m, p, q, nout, ds, &plan, &need)) != DC_OK) return st;
  if ((st = check_work(work, work_bytes, need)) != DC_OK) return st;
  return pq_run(f, g, h, m, p, q, nout, ds, work, work_bytes, (cudaStream_t)stream);
}

static dc_status run_dot2(int32_t pk, int kind, int32_t ndim, const int64_t* dims, const void* f1,
                          const void* g1, const void* f2, const void* g2, void* h, int32_t dtype, void* work,
                          size_t work_bytes, void* stream) {
  if (!dims || ndim < 1 || ndim > 3) return DC_ERR_ARG;
  const void* ins[4] = {f1, g1, f2, g2};
  void* outs[1] = {h};
  if (ndim == 1) return run_1d(kind, ins, 4, outs, 1, dims[0], dtype, work, work_bytes, stream);
  return run_md(pk, ndim, dims, ins, 4, outs, 1, dtype, work, work_bytes, stream);
}

dc_status dc_conv_complex_dot2(int32_t ndim, const int64_t* dims, const void* f1, const void* g1,
                               const void* f2, const void* g2, void* h, int32_t dtype, void* work,
                               size_t work_bytes, void* stream) {
  return run_dot2(DC_KIND_COMPLEX_DOT2, K_COMPLEX_DOT2, ndim, dims, f1, g1, f2, g2, h, dtype, work, work_bytes,
                  stream);
}

dc_status dc_conv_hermitian_dot2(int32_t ndim, const int64_t* dims, const void* f1, const void* g1,
                                 const void* f2, const void* g2, void* h, int32_t dtype, void* work,
                                 size_t work_bytes, void* stream) {
  return run_dot2(DC_KIND_HERMITIAN_DOT2, K_HERMITIAN_DOT2, ndim, dims, f1, g1, f2, g2, h, dtype, work,
                  work_bytes, stream);
}

dc_status dc_conv_ternary_hermitian_2d(const void* f, const void* g, const void* e, void* h, int64_t mx,
                                       int64_t my, int32_t dtype, void* work, size_t work_bytes, void* stream) {
  const void* ins[3] = {f, g, e};
  void* outs[1] = {h};
  const int64_t d[2] = {mx, my};
  return run_md(DC_KIND_TERNARY, 2, d, ins, 3, outs, 1, dtype, work, work_bytes, stream);
}

dc_status dc_conv_ternary_hermitian_3d(const void* f, const void* g, const void* e, void* h, int64_t mx,
                                       int64_t my, int64_t mz, int32_t dtype, void* work, size_t work_bytes,
                                       void* stream) {
  const void* ins[3] = {f, g, e};
  void* outs[1] = {h};
  const int64_t d[3] = {mx, my, mz};
  return run_md(DC_KIND_TERNARY, 3, d, ins, 3, outs, 1, dtype, work, work_bytes, stream);
}

dc_status dc_conv_complex_2d(const void* f, const void* g, void* h, int64_t mx, int64_t my,
                             int32_t dtype, void* work, size_t work_bytes, void* stream) {
  const void* ins[2] = {f, g};
  void* outs[1] = {h};
  const int64_t d[2] = {mx, my};
  return run_md(DC_KIND_COMPLEX, 2, d, ins, 2, outs, 1, dtype, work, work_bytes, stream);
}

dc_status dc_conv_complex_3d(const void* f, const void* g, void* h, int64_t mx, int64_t my,
                             int64_t mz, int32_t dtype, void* work, size_t work_bytes, void* stream) {
  const void* ins[2] = {f, g};
  void* outs[1] = {h};
  const int64_t d[3] = {mx, my, mz};
  return run_md(DC_KIND_COMPLEX, 3, d, ins, 2, outs, 1, dtype, work, work_bytes, stream);
}

dc_status dc_conv_hermitian_2d(const void* f, const void* g, void* h, int64_t mx, int64_t my,
                               int32_t dtype, void* work, size_t work_bytes, void* stream) {
  const void* ins[2] = {f, g};
  void* outs[1] = {h};
  const int64_t d[2] = {mx, my};
  return run_md(DC_KIND_HERMITIAN, 2, d, ins, 2, outs, 1, dtype, work, work_bytes, stream);
}

dc_status dc_conv_hermitian_3d(const void* f, const void* g, void* h, int64_t mx, int64_t my,
                               int64_t mz, int32_t dtype, void* work, size_t work_bytes,
                               void* stream) {
  const void* ins[2] = {f, g};
  void* outs[1] = {h};
  const int64_t d[3] = {mx, my, mz};
  return run_md(DC_KIND_HERMITIAN, 3, d, ins, 2, outs, 1, dtype, work, work_bytes, stream);
}

dc_status dc_conv_complex_2d_adjoint(const void* w, const void* f, const void* g, void* df,
                                     void* dg, int64_t mx, int64_t my, int32_t dtype, void* work,
                                     size_t work_bytes, void* stream) {
  const void* ins[3] = {w, f, g};
  void* outs[2] = {df, dg};
  const int64_t d[2] = {mx, my};
  return run_md(DC_KIND_COMPLEX_ADJOINT, 2, d, ins, 3, outs, 2, dtype, work, work_bytes, stream);
}

dc_status dc_conv_complex_3d_adjoint(const void* w, const void* f, const void* g, void* df,
                                     void* dg, int64_t mx, int64_t my, int64_t mz, int32_t dtype,
                                     void* work, size_t work_bytes, void* stream) {
  const void* ins[3] = {w, f, g};
  void* outs[2] = {df, dg};
  const int64_t d[3] = {mx, my, mz};
  return run_md(DC_KIND_COMPLEX_ADJOINT, 3, d, ins, 3, outs, 2, dtype, work, work_bytes, stream);
}

dc_status dc_conv_hermitian_2d_adjoint(const void* w, const void* f, const void* g, void* df,
                                       void* dg, int64_t mx, int64_t my, int32_t dtype, void* work,
                                       size_t work_bytes, void* stream) {
  const void* ins[3] = {w, f, g};
  void* outs[2] = {df, dg};
  const int64_t d[2] = {mx, my};
  return run_md(DC_KIND_HERMITIAN_ADJOINT, 2, d, ins, 3, outs, 2, dtype, work, work_bytes, stream);
}

dc_status dc_conv_hermitian_3d_adjoint(const void* w, const void* f, const void* g, void* df,
                                       void* dg, int64_t mx, int64_t my, int64_t mz, int32_t dtype,
                                       void* work, size_t work_bytes, void* stream) {
  const void* ins[3] = {w, f, g};
  void* outs[2] = {df, dg};
  const int64_t d[3] = {mx, my, mz};
  return run_md(DC_KIND_HERMITIAN_ADJOINT, 3, d, ins, 3, outs, 2, dtype, work, work_bytes, stream);
}

}  // extern "C"

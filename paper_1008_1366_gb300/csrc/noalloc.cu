// dc_conv_complex_1d_noalloc: the 1D complex convolution for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or ask an allocator for a workspace:
// code running under a CUDA stream capture in global capture mode (where
// cudaMalloc is a prohibited call), code embedded in a host application whose
// device memory is owned by an allocator it may not bypass, and real-time
// loops that cannot afford cudaMalloc's implicit device synchronization.
// This entry point needs only its inputs and outputs: its scratch (the
// workspace status header, the root-of-unity table and one two-level scratch
// slot) lives in one file-scope __device__ array of fixed size, which every
// GPU that loads the library holds until the process exits.
#include <mutex>

#include "conv1d.cuh"
#include "launch.h"
#include "plan.h"
#include "tables.h"

using namespace dc;

namespace {

// 2 MiB: header (256 B) + root table (2m entries) + one scratch slot (4m
// entries) for the largest supported m: 40960 (complex64) or 20480 (complex128).
constexpr size_t kNoAllocBytes = 2u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_mu;
void* g_addr[64] = {nullptr};

// Device address of the array on the current device.  In host code the
// array's name only stands for the symbol, so the address is looked up once
// per device, with that device current.
dc_status scratch_address(void** out) {
  int dev = 0;
  DC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return DC_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    DC_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return DC_OK;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" dc_status dc_conv_complex_1d_noalloc(const void* f, const void* g, void* h, int64_t m,
                                                int32_t dtype, void* stream) {
  const int ds = dtype == DC_C64 ? 8 : dtype == DC_C128 ? 16 : 0;
  if (!ds || m < 1 || !f || !g || !h) return DC_ERR_ARG;
  if ((uintptr_t)f % ds || (uintptr_t)g % ds || (uintptr_t)h % ds) return DC_ERR_ALIGN;
  const size_t bytes = (size_t)m * ds;
  for (const void* in : {f, g}) {
    const char* a = (const char*)h;
    const char* b = (const char*)in;
    if (h != in && a < b + bytes && b < a + bytes) return DC_ERR_ARG;
  }
  CfgDev cfg;
  if (!make_cfg(K_COMPLEX, m, ds, kThreads, device_info().smem_optin - kStaticSmemReserve, 0, &cfg))
    return DC_ERR_SIZE;
  const size_t table = align256((size_t)cfg.TN * ds);
  const size_t slot = align256(cfg_scratch_bytes(K_COMPLEX, cfg, ds));
  if (sizeof(WorkHeader) + table + slot > kNoAllocBytes) return DC_ERR_SIZE;
  void* base = nullptr;
  dc_status st = scratch_address(&base);
  if (st != DC_OK) return st;
  char* b = (char*)base;
  cudaStream_t s = (cudaStream_t)stream;
  // the array keeps the previous call's contents: rebuild the table and
  // clear the status header every call
  if ((st = launch_gen_roots(b + sizeof(WorkHeader), cfg.TN, ds, s)) != DC_OK) return st;
  DC_CUDA_TRY(cudaMemsetAsync(b, 0, sizeof(WorkHeader), s));
  cfg.tw = b + sizeof(WorkHeader);
  ConvArgs a{};
  a.in[0] = f;
  a.in[1] = g;
  a.out[0] = h;
  a.nitems = 1;
  a.ninst = 1;
  a.hdr = (WorkHeader*)b;
  a.scratch = b + sizeof(WorkHeader) + table;
  a.slot_bytes = (int64_t)slot;
  a.cfg0 = cfg;
  return launch_conv1d(K_COMPLEX, ds, a, 1, cfg.smem, s);
}

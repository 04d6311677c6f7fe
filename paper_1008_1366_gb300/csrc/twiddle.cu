// Root-of-unity tables zeta_TN^i = exp(2 pi i * i / TN), i < TN.
//
// The paper forms zeta_N^k on the fly from two short tables, one complex
// multiply per factor (Sec. 2.1).  On GB300 the full table of a size costs a
// few MB of HBM, is L2-resident while in use and needs no multiply, so one
// table per (TN, precision) is generated once per device: in FP64 with
// CUDA's sincospi, then rounded to the working precision.
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "tables.h"

namespace dc {

template <class C>
__global__ void gen_roots_kernel(C* out, int64_t TN) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= TN) return;
  double s, c;
  sincospi(2.0 * (double)i / (double)TN, &s, &c);
  out[i] = mk<C>(c, s);
}

namespace {
std::mutex g_mu;
std::map<std::tuple<int, int64_t, int>, void*> g_tables;
}

dc_status launch_gen_roots(void* out, int64_t TN, int dsize, cudaStream_t s) {
  const int threads = 256;
  const unsigned blocks = (unsigned)((TN + threads - 1) / threads);
  if (dsize == 8) gen_roots_kernel<float2><<<blocks, threads, 0, s>>>((float2*)out, TN);
  else gen_roots_kernel<double2><<<blocks, threads, 0, s>>>((double2*)out, TN);
  DC_CUDA_TRY(cudaGetLastError());
  return DC_OK;
}

dc_status get_root_table(int64_t TN, int dsize, const void** out) {
  int dev = 0;
  DC_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_mu);
  auto key = std::make_tuple(dev, TN, dsize);
  auto it = g_tables.find(key);
  if (it != g_tables.end()) { *out = it->second; return DC_OK; }
  void* p = nullptr;
  DC_CUDA_TRY(cudaMalloc(&p, (size_t)TN * dsize));
  cudaStream_t s;
  DC_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  const int threads = 256;
  const unsigned blocks = (unsigned)((TN + threads - 1) / threads);
  if (dsize == 8) gen_roots_kernel<float2><<<blocks, threads, 0, s>>>((float2*)p, TN);
  else gen_roots_kernel<double2><<<blocks, threads, 0, s>>>((double2*)p, TN);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (e != cudaSuccess) { cudaFree(p); dc_set_last_cuda_error(e); return DC_ERR_CUDA; }
  g_tables[key] = p;
  *out = p;
  return DC_OK;
}

}  // namespace dc

// Instantiations and host launcher of the fused 1D kernels.
#include <mutex>

#include "conv1d.cuh"
#include "launch.h"

namespace dc {

namespace {
std::mutex g_attr_mu;
}

template <int KIND, class C>
static dc_status launch_t(const ConvArgs& a, int grid, int smem, cudaStream_t s) {
  auto kern = conv1d_kernel<KIND, C>;
  {
    // raise the dynamic shared-memory limit once per kernel and device
    static bool done[64] = {false};
    int dev = 0;
    DC_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_attr_mu);
    if (dev < 64 && !done[dev]) {
      DC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       device_info().smem_optin - kStaticSmemReserve));
      done[dev] = true;
    }
  }
  kern<<<grid, kThreads, smem, s>>>(a);
  DC_CUDA_TRY(cudaGetLastError());
  return DC_OK;
}

dc_status launch_conv1d(int kind, int dsize, const ConvArgs& a, int grid, int smem, cudaStream_t s) {
  if (dsize == 8) {
    switch (kind) {
      case K_COMPLEX:       return launch_t<K_COMPLEX, float2>(a, grid, smem, s);
      case K_HERMITIAN:     return launch_t<K_HERMITIAN, float2>(a, grid, smem, s);
      case K_TERNARY:       return launch_t<K_TERNARY, float2>(a, grid, smem, s);
      case K_COMPLEX_ADJ:   return launch_t<K_COMPLEX_ADJ, float2>(a, grid, smem, s);
      case K_HERMITIAN_ADJ: return launch_t<K_HERMITIAN_ADJ, float2>(a, grid, smem, s);
      case K_HERMITIAN_PAIR: return launch_t<K_HERMITIAN_PAIR, float2>(a, grid, smem, s);
    }
  } else {
    switch (kind) {
      case K_COMPLEX:       return launch_t<K_COMPLEX, double2>(a, grid, smem, s);
      case K_HERMITIAN:     return launch_t<K_HERMITIAN, double2>(a, grid, smem, s);
      case K_TERNARY:       return launch_t<K_TERNARY, double2>(a, grid, smem, s);
      case K_COMPLEX_ADJ:   return launch_t<K_COMPLEX_ADJ, double2>(a, grid, smem, s);
      case K_HERMITIAN_ADJ: return launch_t<K_HERMITIAN_ADJ, double2>(a, grid, smem, s);
      case K_HERMITIAN_PAIR: return launch_t<K_HERMITIAN_PAIR, double2>(a, grid, smem, s);
    }
  }
  return DC_ERR_ARG;
}

dc_status conv1d_blocks_per_sm(int kind, int dsize, int smem, int* out) {
  const void* f = nullptr;
#define DC_PICK(K)                                                                      \
  f = dsize == 8 ? (const void*)conv1d_kernel<K, float2> : (const void*)conv1d_kernel<K, double2>
  switch (kind) {
    case K_COMPLEX: DC_PICK(K_COMPLEX); break;
    case K_HERMITIAN: DC_PICK(K_HERMITIAN); break;
    case K_TERNARY: DC_PICK(K_TERNARY); break;
    case K_COMPLEX_ADJ: DC_PICK(K_COMPLEX_ADJ); break;
    case K_HERMITIAN_ADJ: DC_PICK(K_HERMITIAN_ADJ); break;
    case K_HERMITIAN_PAIR: DC_PICK(K_HERMITIAN_PAIR); break;
    default: return DC_ERR_ARG;
  }
#undef DC_PICK
  DC_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   device_info().smem_optin - kStaticSmemReserve));
  int n = 0;
  DC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, kThreads, smem));
  *out = n;
  return DC_OK;
}

}  // namespace dc

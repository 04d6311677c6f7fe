// One instantiation of the fused 1D kernel, for the kind DC_INST_KIND and the
// complex type DC_INST_C (float2 or double2), given on the compiler command
// line.  Compiling each (kind, precision) separately keeps the build parallel.
#include <mutex>

#include "conv1d.cuh"
#include "launch.h"

#ifndef DC_INST_KIND
#error "DC_INST_KIND must be defined"
#endif
#ifndef DC_INST_C
#error "DC_INST_C must be defined"
#endif

#define DC_CAT2(a, b, c) a##b##_##c
#define DC_CAT(a, b, c) DC_CAT2(a, b, c)

namespace dc {

static constexpr int kKind = DC_INST_KIND;
using CInst = DC_INST_C;

static dc_status set_smem_attr() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  DC_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (dev >= 0 && dev < 64 && !done[dev]) {
    DC_CUDA_TRY(cudaFuncSetAttribute(conv1d_kernel<kKind, CInst>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     device_info().smem_optin - kStaticSmemReserve));
    done[dev] = true;
  }
  return DC_OK;
}

dc_status DC_CAT(conv1d_launch_, DC_INST_KIND, DC_INST_TAG)(const ConvArgs& a, int grid, int smem,
                                                            cudaStream_t s) {
  dc_status st = set_smem_attr();
  if (st != DC_OK) return st;
  conv1d_kernel<kKind, CInst><<<grid, kThreads, smem, s>>>(a);
  DC_CUDA_TRY(cudaGetLastError());
  return DC_OK;
}

dc_status DC_CAT(conv1d_occupancy_, DC_INST_KIND, DC_INST_TAG)(int smem, int* out) {
  dc_status st = set_smem_attr();
  if (st != DC_OK) return st;
  int n = 0;
  DC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, conv1d_kernel<kKind, CInst>, kThreads, smem));
  *out = n;
  return DC_OK;
}

}  // namespace dc

// Internal host interfaces between the C ABI layer and the kernel files.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dealias.h"

namespace dc {

struct ConvArgs;

// shared memory kept free for the kernels' static __shared__ variables
constexpr int kStaticSmemReserve = 1024;

struct DeviceInfo {
  int device;
  int sms;
  int smem_optin;   // max dynamic + static shared memory per block (opt-in)
  int l2_bytes;
};
// properties of the current device (cached per device)
const DeviceInfo& device_info();

dc_status launch_conv1d(int kind, int dsize, const ConvArgs& a, int grid, int smem, cudaStream_t s);
dc_status conv1d_blocks_per_sm(int kind, int dsize, int smem, int* out);

}  // namespace dc

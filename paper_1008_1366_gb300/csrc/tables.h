#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

#include "../../include/dealias.h"

namespace dc {
// Device table of zeta_TN^i for i < TN in the given element size (8: float2,
// 16: double2); created on first request per device and kept until exit.
dc_status get_root_table(int64_t TN, int dsize, const void** out);
}  // namespace dc

namespace dc {
// Writes zeta_TN^i, i < TN, into caller-owned device memory on stream s.
dc_status launch_gen_roots(void* out, int64_t TN, int dsize, cudaStream_t s);
}  // namespace dc

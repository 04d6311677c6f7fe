#pragma once
#include <stdint.h>

#include "../../include/dealias.h"

namespace dc {
// Device table of zeta_TN^i for i < TN in the given element size (8: float2,
// 16: double2); created on first request per device and kept until exit.
dc_status get_root_table(int64_t TN, int dsize, const void** out);
}  // namespace dc

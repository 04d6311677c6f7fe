// Dispatch of the fused 1D kernels to their per-(kind, precision)
// instantiations (conv1d_inst.cu compiled once for each).
#include "conv1d.cuh"
#include "launch.h"

namespace dc {

#define DC_DECL(k)                                                                        \
  dc_status conv1d_launch_##k##_f(const ConvArgs&, int, int, cudaStream_t);              \
  dc_status conv1d_launch_##k##_d(const ConvArgs&, int, int, cudaStream_t);              \
  dc_status conv1d_occupancy_##k##_f(int, int*);                                         \
  dc_status conv1d_occupancy_##k##_d(int, int*);
DC_DECL(0)
DC_DECL(1)
DC_DECL(2)
DC_DECL(3)
DC_DECL(4)
DC_DECL(5)
DC_DECL(6)
DC_DECL(7)
#undef DC_DECL

dc_status launch_conv1d(int kind, int dsize, const ConvArgs& a, int grid, int smem, cudaStream_t s) {
  const bool f = dsize == 8;
  switch (kind) {
    case 0: return f ? conv1d_launch_0_f(a, grid, smem, s) : conv1d_launch_0_d(a, grid, smem, s);
    case 1: return f ? conv1d_launch_1_f(a, grid, smem, s) : conv1d_launch_1_d(a, grid, smem, s);
    case 2: return f ? conv1d_launch_2_f(a, grid, smem, s) : conv1d_launch_2_d(a, grid, smem, s);
    case 3: return f ? conv1d_launch_3_f(a, grid, smem, s) : conv1d_launch_3_d(a, grid, smem, s);
    case 4: return f ? conv1d_launch_4_f(a, grid, smem, s) : conv1d_launch_4_d(a, grid, smem, s);
    case 5: return f ? conv1d_launch_5_f(a, grid, smem, s) : conv1d_launch_5_d(a, grid, smem, s);
    case 6: return f ? conv1d_launch_6_f(a, grid, smem, s) : conv1d_launch_6_d(a, grid, smem, s);
    case 7: return f ? conv1d_launch_7_f(a, grid, smem, s) : conv1d_launch_7_d(a, grid, smem, s);
  }
  return DC_ERR_ARG;
}

dc_status conv1d_blocks_per_sm(int kind, int dsize, int smem, int* out) {
  const bool f = dsize == 8;
  switch (kind) {
    case 0: return f ? conv1d_occupancy_0_f(smem, out) : conv1d_occupancy_0_d(smem, out);
    case 1: return f ? conv1d_occupancy_1_f(smem, out) : conv1d_occupancy_1_d(smem, out);
    case 2: return f ? conv1d_occupancy_2_f(smem, out) : conv1d_occupancy_2_d(smem, out);
    case 3: return f ? conv1d_occupancy_3_f(smem, out) : conv1d_occupancy_3_d(smem, out);
    case 4: return f ? conv1d_occupancy_4_f(smem, out) : conv1d_occupancy_4_d(smem, out);
    case 5: return f ? conv1d_occupancy_5_f(smem, out) : conv1d_occupancy_5_d(smem, out);
    case 6: return f ? conv1d_occupancy_6_f(smem, out) : conv1d_occupancy_6_d(smem, out);
    case 7: return f ? conv1d_occupancy_7_f(smem, out) : conv1d_occupancy_7_d(smem, out);
  }
  return DC_ERR_ARG;
}

}  // namespace dc

// Multi-dimensional composition: outer-axis implicit passes (axis.cu) and
// the batched row kernels (conv1d.cuh).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fft.cuh"
#include "../../include/dealias.h"

namespace dc {

constexpr int kAxisQ = 4;   // residue slots per array in AxisArgs

struct AxisArgs {
  const void* in[4];      // backward: arrays to transform (blockIdx.y selects)
  void* out[4 * kAxisQ];  // backward: out[array * kAxisQ + residue], layout (outer, L, inner)
  const void* fin[3 * kAxisQ];   // forward: fin[output * kAxisQ + residue], layout (outer, L, inner)
  void* fout[3];          // forward: outputs, layout (outer, m or 2m-1, inner)
  int64_t outer, inner;
  int64_t proj_mz, proj_ny;   // 3D self-conjugate plane geometry (inner = proj_ny * proj_mz)
  int32_t m;              // unpadded size along the axis
  // 0: complex, q = 2; 1: centered, q = 3; 2: centered ternary (N = 4m) as
  // q = 2 residues of length 2m; 3: centered ternary as q = 4 residues of
  // length m (compile-time axis lengths only, fixed_axis.cu)
  int32_t centered;
  int32_t proj;           // 0: none; 2: 2D column ky = 0; 3: 3D plane kz = 0
  int32_t w;              // columns per block
  int32_t dbl_mask;       // backward arrays whose self-conjugate subspace is U(k) + conj U(-k)
  int32_t halve_mask;     // forward outputs scaled by 1/2 on the self-conjugate subspace
  int32_t TN, pad;
  const void* tw;         // zeta_TN^i, TN = 2m, 3m or 4m
  FftPlan p;              // length-m sub-transform plan
};

// length of the sub-transforms of an axis of unpadded size m
__host__ __device__ inline int axis_len(int centered, int m) { return centered == 2 ? 2 * m : m; }
// residues of an axis mode
__host__ __device__ inline int axis_q(int centered) { return centered == 1 ? 3 : (centered == 3 ? 4 : 2); }
// axis lengths the compile-time outer-axis kernels handle (fixed_axis.cu)
inline bool fixed_axis_len(int64_t m) { return m >= 64 && m <= 4096 && (m & (m - 1)) == 0; }
inline int axis_smem(bool forward, int centered, int m, int w, int ds) {
  const int nout = centered ? 2 * m - 1 : m;
  const int L = axis_len(centered, m);
  return (forward ? (L + nout) : L) * w * ds;
}

dc_status launch_axis(bool forward, int dsize, const AxisArgs& a, int narrays, cudaStream_t s);

// the outer-axis passes on compile-time column transforms (fixed_axis.cu);
// DC_ERR_SIZE for axis lengths that file does not compile
namespace fx {
namespace f32 { dc_status launch_axis_fixed(bool forward, const AxisArgs& a, int narrays, cudaStream_t s); }
namespace f64 { dc_status launch_axis_fixed(bool forward, const AxisArgs& a, int narrays, cudaStream_t s); }
}  // namespace fx

// public multi-D kinds handled by multid.cu
dc_status md_workspace(int pkind, int ndim, const int64_t* dims, int ds, size_t* bytes);
dc_status md_workspace_slabs(int pkind, int ndim, const int64_t* dims, int ds, int64_t slabs, size_t* bytes);
dc_status md_chunking(int pkind, int ndim, const int64_t* dims, int ds, size_t work_bytes, int64_t* slabs,
                      int64_t* chunks);
dc_status md_prepare(int pkind, int ndim, const int64_t* dims, int ds);
dc_status md_run(int pkind, int ndim, const int64_t* dims, int ds, const void* const* ins, int nin,
                 void* const* outs, int nout, void* work, size_t work_bytes, cudaStream_t s);

}  // namespace dc

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

// Uniform batches (n instances of size m at stride m) of the binary complex
// convolution on the fixed-shape engine (batched.cu): whether m qualifies,
// the workspace bytes (host-only), and the cached plan (created on first use).
bool fx_uniform_ok(int64_t m, int ds);
bool fx_uniform_two_level(int64_t m);   // m runs as row/column passes spread over many blocks
// mode: the fixed engine's kind of convolution (fx::MODE_*, 0 = binary complex)
size_t fx_uniform_work(int64_t n, int64_t m, int ds, int mode = 0);
dc_status fx_uniform_plan(int64_t n, int64_t m, int ds, struct dc_batched_plan** out, int mode = 0);
// the rows of a centered Hermitian gradient on a MODE_PAIR plan:
// df = conv(w, g), dg = conv(w, f); outputs may be inputs
dc_status fx_pair_run(struct dc_batched_plan* p, const void* w, const void* f, const void* g, void* df, void* dg,
                      void* work, size_t work_bytes, cudaStream_t s);
// the rows of a dot product of two centered Hermitian pairs on a MODE_HDOT2
// plan: h = f1 * g1 + f2 * g2; h may be an input
dc_status fx_hdot2_run(struct dc_batched_plan* p, const void* f1, const void* g1, const void* f2, const void* g2,
                       void* h, void* work, size_t work_bytes, cudaStream_t s);
// the rows of a centered Hermitian ternary convolution on a MODE_TERN4 plan
// (one-level m, four m-point residues): h = f * g * e; h may be an input
dc_status fx_tern4_run(struct dc_batched_plan* p, const void* f, const void* g, const void* e, void* h,
                       void* work, size_t work_bytes, cudaStream_t s);
// n centered Hermitian ternary convolutions of length m at stride m on the
// fixed engine (2m a two-level size of the set): one 1D call, or the rows of
// a multi-D call; outputs may be inputs
bool fx_ternary_ok(int64_t m, int ds);
size_t fx_ternary_work(int64_t m, int ds, int64_t n = 1);
dc_status fx_ternary_plan(int64_t m, int ds, struct dc_batched_plan** out, int64_t n = 1);
dc_status fx_ternary_run(int64_t m, int ds, const void* f, const void* g, const void* e, void* h, void* work,
                         size_t work_bytes, cudaStream_t s, int64_t n = 1);
dc_status conv1d_blocks_per_sm(int kind, int dsize, int smem, int* out);

// general implicit padding (pq.cu): checks and plans a call (the m-point
// transform, the workspace bytes), and runs it
struct FftPlan;
dc_status pq_plan(int64_t m, int32_t p, int32_t q, int64_t nout, int ds, FftPlan* plan_out, size_t* work);
dc_status pq_run(const void* f, const void* g, void* h, int64_t m, int32_t p, int32_t q, int64_t nout, int ds,
                 void* work, size_t work_bytes, cudaStream_t s);

}  // namespace dc

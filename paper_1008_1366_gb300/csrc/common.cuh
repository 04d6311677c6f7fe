// Shared definitions for the sm_103a kernels of the dealiased-convolution
// library: complex helpers, status codes, launch checks.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dealias.h"

namespace dc {

template <class R> struct CT;
template <> struct CT<float>  { using type = float2; };
template <> struct CT<double> { using type = double2; };
template <class R> using cpx = typename CT<R>::type;

template <class C> __host__ __device__ __forceinline__ C mk(double x, double y) {
  C c; c.x = (decltype(c.x))x; c.y = (decltype(c.y))y; return c;
}
template <class C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <class C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <class C> __device__ __forceinline__ C cmul(C a, C b) {
  C c; c.x = a.x * b.x - a.y * b.y; c.y = a.x * b.y + a.y * b.x; return c;
}
// a * conj(b)
template <class C> __device__ __forceinline__ C cmulc(C a, C b) {
  C c; c.x = a.x * b.x + a.y * b.y; c.y = a.y * b.x - a.x * b.y; return c;
}
template <class C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
// i * a
template <class C> __device__ __forceinline__ C cmuli(C a) { C c; c.x = -a.y; c.y = a.x; return c; }
template <class C, class R> __device__ __forceinline__ C cscale(C a, R s) { a.x *= s; a.y *= s; return a; }
// multiply by the root w or by conj(w) depending on the sign
template <int S, class C> __device__ __forceinline__ C cmul_s(C a, C w) {
  return S > 0 ? cmul(a, w) : cmulc(a, w);
}

// device-side status word (first word of every workspace)
struct WorkHeader {
  int32_t status;     // DC_OK or the first error code a kernel recorded
  int32_t detail;     // kernel-specific detail of that error
  uint32_t counter;   // persistent-queue counter, reset before each launch
  uint32_t waited;    // task-queue kernels: tasks that found a dependency unmet
  unsigned long long wait_cycles;   // and the SM cycles they spent waiting
  unsigned long long type_cycles[4];   // SM cycles spent in tasks of each type
  uint32_t type_count[4];              // and the number of such tasks
  unsigned long long handover_cycles;  // cycles from a task's end to the next one's start (queue, dependency)
  unsigned long long table_cycles;     // cycles spent loading root tables into shared memory
  uint32_t pad[42];
};
static_assert(sizeof(WorkHeader) == 256, "workspace header is 256 bytes");

__device__ __forceinline__ void record_error(WorkHeader* hdr, int code, int detail) {
  if (hdr && atomicCAS(&hdr->status, 0, code) == 0) hdr->detail = detail;
}

}  // namespace dc

#define DC_CUDA_TRY(expr)                                  \
  do {                                                     \
    cudaError_t _e = (expr);                               \
    if (_e != cudaSuccess) { dc_set_last_cuda_error(_e); return DC_ERR_CUDA; } \
  } while (0)

extern "C" void dc_set_last_cuda_error(cudaError_t e);

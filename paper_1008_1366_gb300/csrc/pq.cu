// General implicit padding (Sec. 2.4): p m data modes zero padded to N = q m.
// With j = q l + r (l < m, r < q) and k = t m + s (t < p, s < m),
//   u_{q l + r} = sum_{s<m} zeta_m^{l s} W_r(s),
//   W_r(s)      = sum_{t<p} zeta_{qm}^{r (t m + s)} U_{t m + s},
// so the backward transform of size q m is q transforms of size m of the
// p-term sums W_r; the forward transform
//   q m U_k = sum_{r<q} zeta_{qm}^{-r k} sum_{l<m} zeta_m^{-l k} u_{q l + r}
// is again q transforms of size m, read at s = k mod m for every output
// k < q m (the m-point transform is m-periodic in k).  For the binary
// complex convolution the product u^f u^g is formed between them.
//
// One block per residue r: it forms W_r of f and g in shared memory, runs
// both m-point backward transforms (fft.cuh), the product, the forward
// transform, and writes its twiddled contribution zeta_{qm}^{-rk} S_r(k mod m)
// to every requested output k into the workspace; a second kernel sums the q
// contributions and scales by 1/(q m).  With q >= 2p the outputs k < 2pm - 1
// are the whole linear convolution (p = 1, q = 2: all 2m - 1 of them).
#include <algorithm>

#include "fft.cuh"
#include "launch.h"
#include "plan.h"
#include "tables.h"

namespace dc {
namespace {

constexpr int kPqThreads = 512;
constexpr size_t kHeader = sizeof(WorkHeader);

struct PqArgs {
  const void* f;
  const void* g;
  void* contrib;       // q arrays of nout elements
  const void* tw;      // zeta_{qm}^i, i < q m
  int32_t m, p, q, nout;
  FftPlan plan;        // m-point transform
};

template <class C>
__global__ void __launch_bounds__(kPqThreads) pq_residue_kernel(const __grid_constant__ PqArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* A = reinterpret_cast<C*>(smem_raw);
  C* B = A + a.m;
  const int r = blockIdx.x, m = a.m, TN = a.q * m;
  const C* f = (const C*)a.f;
  const C* g = (const C*)a.g;
  const C* tw = (const C*)a.tw;
  // W_r(s) of both inputs
  for (int s = threadIdx.x; s < m; s += blockDim.x) {
    C wf, wg;
    wf.x = wf.y = 0;
    wg.x = wg.y = 0;
    for (int t = 0; t < a.p; ++t) {
      const int k = t * m + s;
      const C z = __ldg(&tw[(int)(((int64_t)r * k) % TN)]);
      wf = cadd(wf, cmul(__ldg(f + k), z));
      wg = cadd(wg, cmul(__ldg(g + k), z));
    }
    A[s] = wf;
    B[s] = wg;
  }
  __syncthreads();
  const int i = threadIdx.x;
  const bool act = i < a.plan.tpt;
  fft_smem<1>(A, 1, a.plan, i, act, tw, TN);
  fft_smem<1>(B, 1, a.plan, i, act, tw, TN);
  for (int s = threadIdx.x; s < m; s += blockDim.x) A[s] = cmul(A[s], B[s]);
  __syncthreads();
  fft_smem<-1>(A, 1, a.plan, i, act, tw, TN);
  C* out = (C*)a.contrib + (size_t)r * a.nout;
  for (int k = threadIdx.x; k < a.nout; k += blockDim.x)
    out[k] = cmulc(A[k % m], __ldg(&tw[(int)(((int64_t)r * k) % TN)]));   // zeta_{qm}^{-rk}
}

template <class C>
__global__ void pq_sum_kernel(const C* contrib, C* h, int q, int nout, int m) {
  using R = decltype(h[0].x);
  const R sc = (R)1 / (R)((int64_t)q * m);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nout; k += gridDim.x * blockDim.x) {
    C s = contrib[k];
    for (int r = 1; r < q; ++r) s = cadd(s, contrib[(size_t)r * nout + k]);
    h[k] = cscale(s, sc);
  }
}

int pq_smem(int64_t m, int ds) { return (int)(2 * m * ds); }

}  // namespace

// Checks and plans a call; *plan_out gets the m-point plan.
dc_status pq_plan(int64_t m, int32_t p, int32_t q, int64_t nout, int ds, FftPlan* plan_out, size_t* work) {
  if (m < 1 || p < 1 || q < p || q > 16 || nout < 1 || nout > (int64_t)q * m) return DC_ERR_ARG;
  if ((int64_t)q * m > (1 << 24)) return DC_ERR_SIZE;
  if (!make_fft_plan((int)m, ds == 8 ? 30 : 15, plan_out) || plan_out->tpt > kPqThreads) return DC_ERR_SIZE;
  if (pq_smem(m, ds) > device_info().smem_optin - kStaticSmemReserve) return DC_ERR_SIZE;
  *work = kHeader + (size_t)q * nout * ds;
  return DC_OK;
}

dc_status pq_run(const void* f, const void* g, void* h, int64_t m, int32_t p, int32_t q, int64_t nout, int ds,
                 void* work, size_t work_bytes, cudaStream_t s) {
  FftPlan plan;
  size_t need = 0;
  dc_status st = pq_plan(m, p, q, nout, ds, &plan, &need);
  if (st != DC_OK) return st;
  if (work_bytes < need) return DC_ERR_NOMEM;
  PqArgs a{};
  a.f = f;
  a.g = g;
  a.contrib = (char*)work + kHeader;
  a.m = (int32_t)m;
  a.p = p;
  a.q = q;
  a.nout = (int32_t)nout;
  a.plan = plan;
  if ((st = get_root_table((int64_t)q * m, ds, &a.tw)) != DC_OK) return st;
  DC_CUDA_TRY(cudaMemsetAsync(work, 0, kHeader, s));
  const int smem = pq_smem(m, ds);
  const int grid2 = (int)std::min<int64_t>((nout + 255) / 256, 4 * device_info().sms);
  if (ds == 8) {
    DC_CUDA_TRY(cudaFuncSetAttribute(pq_residue_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    pq_residue_kernel<float2><<<q, kPqThreads, smem, s>>>(a);
    pq_sum_kernel<float2><<<grid2, 256, 0, s>>>((const float2*)a.contrib, (float2*)h, q, (int)nout, (int)m);
  } else {
    DC_CUDA_TRY(cudaFuncSetAttribute(pq_residue_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    pq_residue_kernel<double2><<<q, kPqThreads, smem, s>>>(a);
    pq_sum_kernel<double2><<<grid2, 256, 0, s>>>((const double2*)a.contrib, (double2*)h, q, (int)nout, (int)m);
  }
  DC_CUDA_TRY(cudaGetLastError());
  return DC_OK;
}

}  // namespace dc

// Implicitly padded transforms along an outer (strided) axis, for the
// multi-dimensional convolutions (Sec. 3: Functions cconv2, conv2, cconv3 and
// the 3D centered Hermitian case).
//
// Data are (outer, axis, inner) row-major with the inner index contiguous.
// A block owns one outer index and a tile of w consecutive inner indices
// (w columns); it loads the whole axis for those columns (coalesced rows of
// w elements), builds the residue inputs in shared memory, runs the m-point
// sub-transforms down the columns (fft.cuh, interleaved layout) and writes
// the residue arrays.  Kinds:
//   complex  (q = 2): axis holds m values, residue r = 0, 1 input
//            zeta_{2m}^{rk} U_k (Eq. (2.1)); forward Eq. (2.2).
//   centered (q = 3): axis holds 2m-1 values, origin at m-1; residue
//            r = -1, 0, 1 input w_{k,r} of Eqs. (2.4)-(2.5); forward Eq. (2.6)
//            for k = -m+1..m-1.
//   ternary  (q = 2, sub-transforms of length 2m, N = 4m; Sec. 4.1): axis
//            holds 2m-1 values, origin at m-1, U_{-m} = 0; residue r = 0, 1
//            backward u_{2l+r} = sum_k zeta_{2m}^{lk} zeta_{4m}^{rk} U_k, a
//            2m-point transform of zeta_{4m}^{rk} U_k placed at k mod 2m;
//            forward 4m U_k = sum_r zeta_{4m}^{-rk} sum_l zeta_{2m}^{-lk}
//            u_{2l+r} for k = -m+1..m-1 (the transform read at k mod 2m;
//            Eqs. (fft0tbackward)-(fft0tforward) before their index shift).
// Backward writes one array per residue, (outer, L, inner) with L the
// sub-transform length.  Forward reads the q residue arrays and writes the
// recombined, scaled result.
// Hermitian data: the self-conjugate subspace (last-axis wavenumber 0) is
// projected onto U(-k) = conj U(k) while loading (Sec. 5 asks a routine to
// enforce the symmetry); mode `dbl` instead forms U(k) + conj U(-k) there
// (the symmetrized upstream gradient), and forward mode `halve` scales that
// subspace by 1/2 (gradient outputs).
#include "fft.cuh"
#include "launch.h"
#include "multid.h"

namespace dc {

__device__ __forceinline__ bool on_selfconj(const AxisArgs& a, int64_t i, int64_t* mirror) {
  if (a.proj == 2) { *mirror = 0; return i == 0; }                      // 2D: ky = 0 column
  if (a.proj == 3) {                                                    // 3D: kz = 0 plane
    if (i % a.proj_mz) return false;
    const int64_t iy = i / a.proj_mz;
    *mirror = (a.proj_ny - 1 - iy) * a.proj_mz;
    return true;
  }
  return false;
}

template <class C>
__device__ __forceinline__ C load_sym(const AxisArgs& a, const C* in, int64_t o, int nin, int j,
                                      int64_t i, bool dbl) {
  const C v = in[(o * nin + j) * a.inner + i];
  int64_t mi;
  if (!on_selfconj(a, i, &mi)) return v;
  const C u = in[(o * nin + (nin - 1 - j)) * a.inner + mi];
  C s;
  s.x = v.x + u.x;
  s.y = v.y - u.y;
  if (!dbl) { s.x *= (decltype(s.x))0.5; s.y *= (decltype(s.x))0.5; }
  return s;
}

template <class C>
__global__ void __launch_bounds__(512) axis_backward_kernel(AxisArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int z = blockIdx.y;
  const C* in = (const C*)a.in[z];
  const bool dbl = (a.dbl_mask >> z) & 1;
  const int w = a.w, m = a.m;
  const int64_t tiles_per_outer = (a.inner + w - 1) / w;
  const int64_t o = blockIdx.x / tiles_per_outer;
  const int64_t i0 = (blockIdx.x - o * tiles_per_outer) * w;
  const int T = blockDim.x, tid = threadIdx.x;
  const C* tw = (const C*)a.tw;
  const bool tern = a.centered == 2;
  const int q = a.centered == 1 ? 3 : 2;
  const int nin = a.centered ? 2 * m - 1 : m;
  const int L = axis_len(a.centered, m);
  const int cc = tid % w, ci = tid / w;
  const bool act = ci < a.p.tpt;
  using R = decltype(sm[0].x);
  for (int ri = 0; ri < q; ++ri) {
    const int r = a.centered == 1 ? ri - 1 : ri;
    for (int e = tid; e < L * w; e += T) {
      const int k = e / w, c = e - k * w;
      const int64_t i = i0 + c;
      C v; v.x = 0; v.y = 0;
      if (i < a.inner) {
        if (tern) {
          // transform index k holds wavenumber k (k < m) or k - 2m (k > m);
          // k = m is the zero U_{-m}
          const int kw = k < m ? k : k - 2 * m;
          if (k != m) {
            v = load_sym(a, in, o, nin, kw + m - 1, i, dbl);
            if (r && kw) {
              const C t = __ldg(&tw[kw > 0 ? kw : -kw]);   // zeta_{4m}^{|k|}
              v = kw > 0 ? cmul(v, t) : cmulc(v, t);
            }
          }
        } else if (!a.centered) {
          v = load_sym(a, in, o, nin, k, i, dbl);
          if (r) v = cmul(v, __ldg(&tw[k]));
        } else {
          // w_{k,r} = U_0 at k = 0, else zeta_{3m}^{rk} (U_k + zeta_3^{-r} U_{k-m})
          v = load_sym(a, in, o, nin, k + m - 1, i, dbl);
          if (k > 0) {
            C u = load_sym(a, in, o, nin, k - 1, i, dbl);
            if (r == 0) {
              v = cadd(v, u);
            } else {
              C z3; z3.x = (R)-0.5; z3.y = (R)(-r) * (R)0.86602540378443864676;
              v = cadd(v, cmul(u, z3));
              const C t = __ldg(&tw[k]);
              v = r > 0 ? cmul(v, t) : cmulc(v, t);
            }
          }
        }
      }
      sm[e] = v;
    }
    __syncthreads();
    fft_smem<1>(sm + cc, w, a.p, ci, act, tw, a.TN);
    C* out = (C*)a.out[z * kAxisQ + ri];
    for (int e = tid; e < L * w; e += T) {
      const int k = e / w, c = e - k * w;
      const int64_t i = i0 + c;
      if (i < a.inner) out[(o * L + k) * a.inner + i] = sm[e];
    }
    __syncthreads();
  }
}

template <class C>
__global__ void __launch_bounds__(512) axis_forward_kernel(AxisArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int z = blockIdx.y;
  const int w = a.w, m = a.m;
  const int nout = a.centered ? 2 * m - 1 : m;
  const bool tern = a.centered == 2;
  const int L = axis_len(a.centered, m);
  C* H = sm + (size_t)L * w;
  const int64_t tiles_per_outer = (a.inner + w - 1) / w;
  const int64_t o = blockIdx.x / tiles_per_outer;
  const int64_t i0 = (blockIdx.x - o * tiles_per_outer) * w;
  const int T = blockDim.x, tid = threadIdx.x;
  const C* tw = (const C*)a.tw;
  const int q = a.centered == 1 ? 3 : 2;
  const int cc = tid % w, ci = tid / w;
  const bool act = ci < a.p.tpt;
  using R = decltype(sm[0].x);
  for (int ri = 0; ri < q; ++ri) {
    const int r = a.centered == 1 ? ri - 1 : ri;
    const C* src = (const C*)a.fin[z * kAxisQ + ri];
    for (int e = tid; e < L * w; e += T) {
      const int k = e / w, c = e - k * w;
      const int64_t i = i0 + c;
      C v; v.x = 0; v.y = 0;
      if (i < a.inner) v = src[(o * L + k) * a.inner + i];
      sm[e] = v;
    }
    __syncthreads();
    fft_smem<-1>(sm + cc, w, a.p, ci, act, tw, a.TN);
    for (int e = tid; e < nout * w; e += T) {
      const int j = e / w, c = e - j * w;
      const int k = a.centered ? j - (m - 1) : j;       // wavenumber of output row j
      const int kk = k < 0 ? k + L : k;                  // index of the L-periodic sub-transform
      C x = sm[kk * w + c];
      if (r != 0) {
        // zeta_{qm}^{-rk}
        const int ak = k < 0 ? -k : k;
        const C t = __ldg(&tw[ak]);
        const bool conj_t = (r > 0) == (k >= 0);
        x = conj_t ? cmulc(x, t) : cmul(x, t);
      }
      H[e] = ri ? cadd(H[e], x) : x;
    }
    __syncthreads();
  }
  C* out = (C*)a.fout[z];
  const R scale = (R)1 / (R)(tern ? 4 * m : q * m);
  const bool halve = (a.halve_mask >> z) & 1;
  for (int e = tid; e < nout * w; e += T) {
    const int j = e / w, c = e - j * w;
    const int64_t i = i0 + c;
    if (i < a.inner) {
      R s = scale;
      int64_t mi;
      if (halve && on_selfconj(a, i, &mi)) s *= (R)0.5;
      out[(o * nout + j) * a.inner + i] = cscale(H[e], s);
    }
  }
}

dc_status launch_axis(bool forward, int dsize, const AxisArgs& a, int narrays, cudaStream_t s) {
  // axis lengths with compile-time code (fixed_axis.cu) run there
  const dc_status fst = dsize == 8 ? fx::f32::launch_axis_fixed(forward, a, narrays, s)
                                   : fx::f64::launch_axis_fixed(forward, a, narrays, s);
  if (fst != DC_ERR_SIZE || a.centered == 3) return fst;   // four residues: compile-time lengths only
  const int64_t tiles = a.outer * ((a.inner + a.w - 1) / a.w);
  if (tiles < 1 || narrays < 1) return DC_OK;
  if (tiles > 0x7fffffff) return DC_ERR_SIZE;
  const int smem = axis_smem(forward, a.centered, a.m, a.w, dsize);
  dim3 grid((unsigned)tiles, (unsigned)narrays);
  const int cap = device_info().smem_optin - kStaticSmemReserve;
  if (dsize == 8) {
    auto k = forward ? axis_forward_kernel<float2> : axis_backward_kernel<float2>;
    DC_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    k<<<grid, 512, smem, s>>>(a);
  } else {
    auto k = forward ? axis_forward_kernel<double2> : axis_backward_kernel<double2>;
    DC_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    k<<<grid, 512, smem, s>>>(a);
  }
  DC_CUDA_TRY(cudaGetLastError());
  return DC_OK;
}

}  // namespace dc

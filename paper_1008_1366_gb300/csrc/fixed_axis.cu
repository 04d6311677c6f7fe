// Outer-axis implicit transforms of the multi-dimensional convolutions on
// the fixed-shape column transforms (fixed.cuh), for axis lengths m = 2^a,
// 64 <= m <= 4096.  Same contract as axis.cu (Sec. 3: Functions cconv2,
// conv2, cconv3 and the 3D centered Hermitian case):
//   complex  (q = 2): residue r = 0, 1 input zeta_{2m}^{rk} U_k (Eq. (2.1)),
//            forward recombination Eq. (2.2);
//   centered (q = 3): axis holds 2m-1 values, origin at m-1; residue
//            r = -1, 0, 1 input w_{k,r} of Eqs. (2.4)-(2.5); forward Eq. (2.6)
//            for k = -m+1..m-1.
//   ternary  (q = 4, N = 4m of Sec. 4.1 as four m-point residues): axis as
//            the centered one, U_{-m} = 0; residue r = 0..3 input
//            zeta_{4m}^{rk} (U_k + zeta_4^{-r} U_{k-m}) (U_0 at k = 0);
//            forward: S_r(kk) zeta_{4m}^{-r kk} at k = kk and that times
//            i^r at k = kk - m, summed over r and scaled by 1/(4m).
// A block of NT threads (256; 512 for complex axes of 2048 points and more)
// owns one outer index and a tile of W consecutive inner indices (columns);
// W = NT E / m, T = m / E threads per column.
// Complex axes take E = 16; centered axes, whose tiles also hold the 2m-1
// staged input rows, take E = 8 up to m = 512 (half the columns, half the
// shared memory, twice the resident blocks), where a tile row still fills
// whole 32-byte sectors (W >= 4); at m = 1024 that halving cost more in
// half-used sectors than it gained (2D 1024^2: 0.208 -> 0.228 ms).
// Every stage is compile-time code on registers (no runtime plan), the
// input columns are read once for all residues, and the forward direction
// recombines the residues in shared memory before one scaled write.
// Hermitian data: the self-conjugate subspace is projected while loading
// (or doubled for an upstream gradient, `dbl`), and forward outputs of
// gradients are halved there (`halve`), as in axis.cu.
#include "fixed.cuh"
#include "launch.h"
#include "multid.h"

namespace dc {
namespace fx {
namespace DC_FX_P {

namespace {

// Q residues: 2 complex (N = 2m), 3 centered (N = 3m), 4 the ternary
// kind's N = 4m taken as four m-point residues (below).  Complex axes of
// 2048 and more points run blocks of 512 threads, so that a tile row spans
// W >= 2 (FP32: 4) columns and its loads use whole 32-byte sectors; so do
// the FP32 four-residue axes there (their staged rows still fit); the
// centered ones keep 256.
template <int L, int Q> struct AxisShape {
  static constexpr bool CEN = Q >= 3;
  static constexpr int NT = L >= 2048 && (Q == 2 || (Q == 4 && !kDouble)) ? 512 : kThreads;
  static constexpr int E = CEN && L <= 512 ? 8 : 16;
  static constexpr int T = L / E;
  static constexpr int W = NT * E / L;
  static_assert(L % E == 0 && W >= 1 && W * T == NT, "axis tile covers the block");
};

__host__ __device__ constexpr int axis_ceil_log2(int x) {
  int l = 0;
  while ((1 << l) < x) ++l;
  return l;
}

// shared memory: roots, transform buffer (W L), and for centered axes the
// staged input or recombination buffer ((2m-1) W)
template <int L, int Q> constexpr int axis_smem_bytes() {
  using S = AxisShape<L, Q>;
  return (kRootsMax + S::W * L + (S::CEN ? (2 * L - 1) * S::W : 0)) * (int)sizeof(C);
}

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

// element v of a column on the self-conjugate set, with u the element at
// its mirror (row nin-1-j of the mirror column): projected onto (or, dbl,
// doubled into) the Hermitian-symmetric subspace, (v + conj u) / 2
__device__ __forceinline__ C sym_part(C v, C u, bool dbl) {
  C s;
  s.x = v.x + u.x;
  s.y = v.y - u.y;
  if (!dbl) {
    s.x *= (Real)0.5;
    s.y *= (Real)0.5;
  }
  return s;
}

template <int TN, int NT>
__device__ __forceinline__ Roots<C> fill_roots(const AxisArgs& a, C* rts) {
  constexpr int sh = (axis_ceil_log2(TN) + 1) / 2, nlo = 1 << sh;
  constexpr int cnt = nlo + (TN + nlo - 1) / nlo;
  static_assert(cnt <= kRootsMax, "root tables fit their reservation");
  const C* tab = (const C*)a.tw;
  for (int e = threadIdx.x; e < cnt; e += NT) rts[e] = __ldg(tab + (e < nlo ? e : (e - nlo) << sh));
  __syncthreads();
  return Roots<C>{rts, rts + nlo, sh, nlo - 1};
}

template <int L, int Q>
__global__ void __launch_bounds__(AxisShape<L, Q>::NT) axis_bwd_kernel(const __grid_constant__ AxisArgs a) {
  using S = AxisShape<L, Q>;
  constexpr bool CEN = S::CEN;
  constexpr int E = S::E, W = S::W, TN = Q * L, nin = CEN ? 2 * L - 1 : L;
  using K = Stage<L, E, 0, false>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* rts = (C*)smem_raw;
  C* buf = rts + kRootsMax;
  C* stg = buf + W * L;   // centered: the staged input tile, nin rows of W
  const Roots<C> rt = fill_roots<TN, S::NT>(a, rts);
  const int z = blockIdx.y;
  const C* in = (const C*)a.in[z];
  const bool dbl = (a.dbl_mask >> z) & 1;
  const int64_t tiles = (a.inner + W - 1) / W;
  const int64_t o = blockIdx.x / tiles;
  const int64_t i0 = (blockIdx.x - o * tiles) * W;
  const int c = threadIdx.x % W, i = threadIdx.x / W;
  const int64_t col = i0 + c;
  const bool act = col < a.inner;
  C zero;
  zero.x = 0;
  zero.y = 0;
  if constexpr (!CEN) {
    // the column is read once; residue 1 multiplies it by zeta_{2m}^k
    C raw[E];
    const C* base = in + o * (int64_t)nin * a.inner;
#pragma unroll
    for (int b = 0; b < K::NB; ++b)
#pragma unroll
      for (int q = 0; q < K::R; ++q)
        raw[b * K::R + q] = act ? base[(int64_t)pos<L, E, 0, false>(i, b, q) * a.inner + col] : zero;
    int64_t mi = 0;
    if (act && on_selfconj(a, col, &mi)) {
#pragma unroll
      for (int b = 0; b < K::NB; ++b)
#pragma unroll
        for (int q = 0; q < K::R; ++q)
          raw[b * K::R + q] = sym_part(raw[b * K::R + q],
                                       base[(int64_t)(nin - 1 - pos<L, E, 0, false>(i, b, q)) * a.inner + mi], dbl);
    }
#pragma unroll 1
    for (int r = 0; r < 2; ++r) {
      C v[E];
#pragma unroll
      for (int b = 0; b < K::NB; ++b)
#pragma unroll
        for (int q = 0; q < K::R; ++q) {
          const int e = b * K::R + q;
          v[e] = r ? cmul(raw[e], rt.at(pos<L, E, 0, false>(i, b, q))) : raw[e];
        }
      C* out = (C*)a.out[z * kAxisQ + r] + o * (int64_t)L * a.inner + col;
      column<L, E, W, TN, false>(v, i, buf + c, rt, [&](int j, int, C y) {
        if (act) out[(int64_t)j * a.inner] = y;
      });
      __syncthreads();
    }
  } else {
    // stage the 2m-1 stored rows of the tile once (coalesced rows of W).  A
    // thread keeps its column c for every row it stages, so the test for
    // the self-conjugate set is made once, and the loads of its rows are
    // independent of one another.
    {
      static_assert(S::NT % W == 0, "a thread keeps its column while staging");
      int64_t mi = 0;
      const bool sym = act && on_selfconj(a, col, &mi);
      const C* base = in + o * (int64_t)nin * a.inner;
#pragma unroll 8
      for (int j = i; j < nin; j += S::NT / W) {
        C v = act ? base[(int64_t)j * a.inner + col] : zero;
        if (sym) v = sym_part(v, base[(int64_t)(nin - 1 - j) * a.inner + mi], dbl);
        stg[j * W + c] = v;
      }
    }
    __syncthreads();
#pragma unroll 1
    for (int ri = 0; ri < Q; ++ri) {
      const int r = Q == 3 ? ri - 1 : ri;
      C v[E];
#pragma unroll
      for (int b = 0; b < K::NB; ++b)
#pragma unroll
        for (int q = 0; q < K::R; ++q) {
          // w_{k,r} = U_0 at k = 0, else zeta_{Qm}^{rk} (U_k + zeta_Q^{-r} U_{k-m})
          // (Q = 4: the ternary kind's U_{-m} = 0, so k = 0 holds U_0 alone)
          const int k = pos<L, E, 0, false>(i, b, q);
          C x = stg[(k + L - 1) * W + c];
          if (k > 0) {
            const C u = stg[(k - 1) * W + c];
            if (r == 0) {
              x = cadd(x, u);
            } else if constexpr (Q == 3) {
              C z3;
              z3.x = (Real)-0.5;
              z3.y = (Real)(-r) * (Real)0.86602540378443864676;
              x = cadd(x, cmul(u, z3));
              const C t = rt.at(k);
              x = r > 0 ? cmul(x, t) : cmulc(x, t);
            } else {
              // zeta_4^{-r} = (-i)^r
              C z;
              z.x = r == 1 ? u.y : (r == 2 ? -u.x : -u.y);
              z.y = r == 1 ? -u.x : (r == 2 ? -u.y : u.x);
              x = cmul(cadd(x, z), rt.at(r * k));
            }
          }
          v[b * K::R + q] = x;
        }
      C* out = (C*)a.out[z * kAxisQ + ri] + o * (int64_t)L * a.inner + col;
      column<L, E, W, TN, false>(v, i, buf + c, rt, [&](int j, int, C y) {
        if (act) out[(int64_t)j * a.inner] = y;
      });
      __syncthreads();
    }
  }
}

template <int L, int Q>
__global__ void __launch_bounds__(AxisShape<L, Q>::NT) axis_fwd_kernel(const __grid_constant__ AxisArgs a) {
  using S = AxisShape<L, Q>;
  constexpr bool CEN = S::CEN;
  constexpr int E = S::E, W = S::W, q = Q, TN = q * L, nout = CEN ? 2 * L - 1 : L;
  using K = Stage<L, E, 0, true>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* rts = (C*)smem_raw;
  C* buf = rts + kRootsMax;
  C* H = buf + W * L;   // centered: the recombined outputs, nout rows of W
  const Roots<C> rt = fill_roots<TN, S::NT>(a, rts);
  const int z = blockIdx.y;
  const int64_t tiles = (a.inner + W - 1) / W;
  const int64_t o = blockIdx.x / tiles;
  const int64_t i0 = (blockIdx.x - o * tiles) * W;
  const int c = threadIdx.x % W, i = threadIdx.x / W;
  const int64_t col = i0 + c;
  const bool act = col < a.inner;
  const Real scale = (Real)1 / (Real)(q * L);
  int64_t mi;
  const bool halve = ((a.halve_mask >> z) & 1) && act && on_selfconj(a, col, &mi);
  const Real sc = halve ? scale * (Real)0.5 : scale;
  C zero;
  zero.x = 0;
  zero.y = 0;
  if constexpr (!CEN) {
    // both residues' columns in registers; residue 0's output stays there
    C vin[2][E];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const C* src = (const C*)a.fin[z * kAxisQ + r] + o * (int64_t)L * a.inner + col;
#pragma unroll
      for (int b = 0; b < K::NB; ++b)
#pragma unroll
        for (int qq = 0; qq < K::R; ++qq)
          vin[r][b * K::R + qq] = act ? src[(int64_t)pos<L, E, 0, true>(i, b, qq) * a.inner] : zero;
    }
    C y0[E];
    column<L, E, W, TN, true>(vin[0], i, buf + c, rt, [&](int, int e, C y) { y0[e] = y; });
    __syncthreads();
    C* out = (C*)a.fout[z] + o * (int64_t)L * a.inner + col;
    column<L, E, W, TN, true>(vin[1], i, buf + c, rt, [&](int k, int e, C y) {
      // Eq. (2.2): (S_0(k) + zeta_{2m}^{-k} S_1(k)) / 2m
      if (act) out[(int64_t)k * a.inner] = cscale(cadd(y0[e], cmulc(y, rt.at(k))), sc);
    });
  } else {
#pragma unroll 1
    for (int ri = 0; ri < Q; ++ri) {
      const int r = Q == 3 ? ri - 1 : ri;
      const C* src = (const C*)a.fin[z * kAxisQ + ri] + o * (int64_t)L * a.inner + col;
      C v[E];
#pragma unroll
      for (int b = 0; b < K::NB; ++b)
#pragma unroll
        for (int qq = 0; qq < K::R; ++qq)
          v[b * K::R + qq] = act ? src[(int64_t)pos<L, E, 0, true>(i, b, qq) * a.inner] : zero;
      // S_r(kk) serves the outputs k = kk (row kk + m - 1) and, for kk > 0,
      // k = kk - m (row kk - 1), each times zeta_{3m}^{-rk} (Eq. (2.6)); the
      // thread owning kk is the same for every residue
      column<L, E, W, TN, true>(v, i, buf + c, rt, [&](int kk, int, C y) {
        C hi = y, lo = y;
        if (r != 0) {
          if constexpr (Q == 3) {
            // k = kk >= 0: zeta_{3m}^{-r kk}; k = kk - m < 0: zeta_{3m}^{-r (kk - m)}
            const C t = rt.at(kk);
            hi = r > 0 ? cmulc(y, t) : cmul(y, t);
            const C u = rt.at(L - kk);
            lo = r > 0 ? cmul(y, u) : cmulc(y, u);
          } else {
            // k = kk: zeta_{4m}^{-r kk}; k = kk - m: that times zeta_4^r = i^r
            hi = cmulc(y, rt.at(r * kk));
            lo.x = r == 1 ? -hi.y : (r == 2 ? -hi.x : hi.y);
            lo.y = r == 1 ? hi.x : (r == 2 ? -hi.y : -hi.x);
          }
        }
        C* h1 = &H[(kk + L - 1) * W + c];
        *h1 = ri ? cadd(*h1, hi) : hi;
        if (kk > 0) {
          C* h0 = &H[(kk - 1) * W + c];
          *h0 = ri ? cadd(*h0, lo) : lo;
        }
      });
      __syncthreads();
    }
    // one scaled write of the tile (coalesced rows of W); a thread keeps its
    // column, whose scale sc was set above
    static_assert(S::NT % W == 0, "a thread keeps its column while writing");
    C* out = (C*)a.fout[z] + o * (int64_t)nout * a.inner + col;
    if (act) {
#pragma unroll 8
      for (int j = i; j < nout; j += S::NT / W) out[(int64_t)j * a.inner] = cscale(H[j * W + c], sc);
    }
  }
}

template <int L, int Q>
dc_status launch_LC(bool forward, const AxisArgs& a, int narrays, cudaStream_t s) {
  using S = AxisShape<L, Q>;
  const int64_t tiles = a.outer * ((a.inner + S::W - 1) / S::W);
  if (tiles < 1 || narrays < 1) return DC_OK;
  if (tiles > 0x7fffffff) return DC_ERR_SIZE;
  constexpr int smem = axis_smem_bytes<L, Q>();
  dim3 grid((unsigned)tiles, (unsigned)narrays);
  auto k = forward ? axis_fwd_kernel<L, Q> : axis_bwd_kernel<L, Q>;
  DC_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  k<<<grid, S::NT, smem, s>>>(a);
  DC_CUDA_TRY(cudaGetLastError());
  return DC_OK;
}

template <int L>
dc_status launch_L(bool forward, const AxisArgs& a, int narrays, cudaStream_t s) {
  if (a.centered == 3) return launch_LC<L, 4>(forward, a, narrays, s);
  return a.centered ? launch_LC<L, 3>(forward, a, narrays, s) : launch_LC<L, 2>(forward, a, narrays, s);
}

}  // namespace

// DC_ERR_SIZE when the axis length is not one this file compiles
dc_status launch_axis_fixed(bool forward, const AxisArgs& a, int narrays, cudaStream_t s) {
  if (a.centered == 2) return DC_ERR_SIZE;   // two 2m-point residues: the runtime-shaped kernels (axis.cu)
  switch (a.m) {
    case 64: return launch_L<64>(forward, a, narrays, s);
    case 128: return launch_L<128>(forward, a, narrays, s);
    case 256: return launch_L<256>(forward, a, narrays, s);
    case 512: return launch_L<512>(forward, a, narrays, s);
    case 1024: return launch_L<1024>(forward, a, narrays, s);
    case 2048: return launch_L<2048>(forward, a, narrays, s);
    case 4096: return launch_L<4096>(forward, a, narrays, s);
    default: return DC_ERR_SIZE;
  }
}

}  // namespace DC_FX_P
}  // namespace fx
}  // namespace dc

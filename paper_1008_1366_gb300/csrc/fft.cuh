// Shared-memory sub-transform engine.
//
// The implicit method replaces every zero-padded DFT of size qm by q DFTs of
// size m (Eqs. (2.1)-(2.2), Sec. 2.2, Sec. 4.1); this file supplies those
// m-point DFTs.  Convention of Sec. 2.1: the backward transform is
// u_j = sum_k zeta_N^{jk} U_k (sign S = +1), the forward transform uses
// zeta_N^{-jk} (S = -1), both unnormalized.
//
// Structure: a Stockham autosort transform, natural order in and out, over a
// runtime list of radices in {2,3,4,5,8,16}.  Each stage is done in place in
// shared memory: every thread first loads the E elements of its E/R
// butterflies into registers, the block synchronizes, then the thread applies
// the stage twiddles, the radix-R butterflies and stores.  E (elements per
// thread) is a compile-time constant that every radix of the plan divides.
// Twiddles come from a table of zeta_TN^i, i < TN, that the host generated in
// FP64 (twiddle.cu); a stage of radix R after Ns points uses
// zeta_{Ns R}^{q k} = table[q k TN / (Ns R)].
#pragma once

#include "common.cuh"

namespace dc {

constexpr int kMaxStages = 16;

struct FftPlan {
  int32_t L;              // transform length
  int32_t E;              // elements per thread (multiple of every radix)
  int32_t tpt;            // threads per transform = L / E
  int32_t ns;             // number of stages
  int8_t r[kMaxStages];   // radices, applied in order
};

// --- radix butterflies: y_k = sum_j x_j zeta_R^{S jk} -----------------------

template <int S, class C> __device__ __forceinline__ void dft2(C& a, C& b) {
  C t = a; a = cadd(t, b); b = csub(t, b);
}

// multiply by S*i
template <int S, class C> __device__ __forceinline__ C mul_si(C a) {
  return S > 0 ? cmuli(a) : cconj(cmuli(cconj(a)));
}

template <int S, class C> __device__ __forceinline__ void dft4(C& x0, C& x1, C& x2, C& x3) {
  C t0 = cadd(x0, x2), t1 = csub(x0, x2);
  C t2 = cadd(x1, x3), t3 = mul_si<S>(csub(x1, x3));
  x0 = cadd(t0, t2); x2 = csub(t0, t2);
  x1 = cadd(t1, t3); x3 = csub(t1, t3);
}

// multiply by (c + S i s)
template <int S, class C, class R> __device__ __forceinline__ C mul_cs(C a, R c, R s) {
  C w; w.x = c; w.y = S > 0 ? s : -s; return cmul(a, w);
}

template <int S, class C> __device__ __forceinline__ void dft8(C* x) {
  using R = decltype(x[0].x);
  const R h = (R)0.70710678118654752440;  // cos(pi/4)
  // even / odd index halves: DFT4 each, then combine with zeta_8^{S k}
  dft4<S>(x[0], x[2], x[4], x[6]);
  dft4<S>(x[1], x[3], x[5], x[7]);
  C o1 = mul_cs<S>(x[3], h, h);
  C o2 = mul_si<S>(x[5]);
  C o3 = mul_cs<S>(x[7], -h, h);
  C e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
  x[0] = cadd(e0, x[1]); x[4] = csub(e0, x[1]);
  x[1] = cadd(e1, o1);   x[5] = csub(e1, o1);
  x[2] = cadd(e2, o2);   x[6] = csub(e2, o2);
  x[3] = cadd(e3, o3);   x[7] = csub(e3, o3);
}

template <int S, class C> __device__ __forceinline__ void dft16(C* x) {
  using R = decltype(x[0].x);
  C e[8], o[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) { e[j] = x[2 * j]; o[j] = x[2 * j + 1]; }
  dft8<S>(e);
  dft8<S>(o);
  // zeta_16^{k} = (cos(pi k / 8), sin(pi k / 8))
  const R c1 = (R)0.92387953251128675613, s1 = (R)0.38268343236508977173;
  const R h = (R)0.70710678118654752440;
  o[1] = mul_cs<S>(o[1], c1, s1);
  o[2] = mul_cs<S>(o[2], h, h);
  o[3] = mul_cs<S>(o[3], s1, c1);
  o[4] = mul_si<S>(o[4]);
  o[5] = mul_cs<S>(o[5], -s1, c1);
  o[6] = mul_cs<S>(o[6], -h, h);
  o[7] = mul_cs<S>(o[7], -c1, s1);
#pragma unroll
  for (int k = 0; k < 8; ++k) { x[k] = cadd(e[k], o[k]); x[k + 8] = csub(e[k], o[k]); }
}

template <int S, class C> __device__ __forceinline__ void dft3(C* x) {
  using R = decltype(x[0].x);
  const R s = (R)0.86602540378443864676;  // sin(2 pi / 3)
  C t = cadd(x[1], x[2]);
  C d = mul_si<S>(csub(x[1], x[2]));
  C a; a.x = x[0].x - (R)0.5 * t.x; a.y = x[0].y - (R)0.5 * t.y;
  x[0] = cadd(x[0], t);
  x[1].x = a.x + s * d.x; x[1].y = a.y + s * d.y;
  x[2].x = a.x - s * d.x; x[2].y = a.y - s * d.y;
}

template <int S, class C> __device__ __forceinline__ void dft5(C* x) {
  using R = decltype(x[0].x);
  const R c1 = (R)0.30901699437494742410;   // cos(2 pi / 5)
  const R c2 = (R)-0.80901699437494742410;  // cos(4 pi / 5)
  const R s1 = (R)0.95105651629515357212;   // sin(2 pi / 5)
  const R s2 = (R)0.58778525229247312917;   // sin(4 pi / 5)
  C t1 = cadd(x[1], x[4]), t2 = cadd(x[2], x[3]);
  C d1 = csub(x[1], x[4]), d2 = csub(x[2], x[3]);
  C a1, a2, b1, b2;
  a1.x = x[0].x + c1 * t1.x + c2 * t2.x; a1.y = x[0].y + c1 * t1.y + c2 * t2.y;
  a2.x = x[0].x + c2 * t1.x + c1 * t2.x; a2.y = x[0].y + c2 * t1.y + c1 * t2.y;
  C u1; u1.x = s1 * d1.x + s2 * d2.x; u1.y = s1 * d1.y + s2 * d2.y;
  C u2; u2.x = s2 * d1.x - s1 * d2.x; u2.y = s2 * d1.y - s1 * d2.y;
  b1 = mul_si<S>(u1); b2 = mul_si<S>(u2);
  x[0] = cadd(x[0], cadd(t1, t2));
  x[1] = cadd(a1, b1); x[4] = csub(a1, b1);
  x[2] = cadd(a2, b2); x[3] = csub(a2, b2);
}

template <int R, int S, class C> __device__ __forceinline__ void dft(C* x) {
  if constexpr (R == 2) dft2<S>(x[0], x[1]);
  else if constexpr (R == 3) dft3<S>(x);
  else if constexpr (R == 4) dft4<S>(x[0], x[1], x[2], x[3]);
  else if constexpr (R == 5) dft5<S>(x);
  else if constexpr (R == 8) dft8<S>(x);
  else if constexpr (R == 16) dft16<S>(x);
}

// --- one Stockham stage, in place in shared memory ----------------------------
// Element idx of this thread's transform lives at base[idx * es].  Thread i of
// the tpt threads of the transform owns butterflies j = i + b*tpt, b < E/R.
// Stage with Ns points done so far: inputs x[j + q L/R], outputs at
// (j - k) R + k + q Ns with k = j mod Ns, after twiddling input q by
// zeta_{Ns R}^{S q k}.
template <int R, int E, int S, class C>
__device__ __forceinline__ void fft_stage(C* base, int es, int L, int Ns, int i, int tpt,
                                          bool active, const C* __restrict__ tw, int tstride) {
  constexpr int NB = E / R;
  C v[E];
  const int LR = L / R;
  if (active) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = i + b * tpt;
#pragma unroll
      for (int q = 0; q < R; ++q) v[b * R + q] = base[(j + q * LR) * es];
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = i + b * tpt;
      const int k = j % Ns;
      if (Ns > 1) {
        const int step = k * tstride;
#pragma unroll
        for (int q = 1; q < R; ++q) v[b * R + q] = cmul_s<S>(v[b * R + q], __ldg(&tw[q * step]));
      }
      dft<R, S>(&v[b * R]);
      const int o = (j - k) * R + k;
#pragma unroll
      for (int q = 0; q < R; ++q) base[(o + q * Ns) * es] = v[b * R + q];
    }
  }
  __syncthreads();
}

template <int E, int S, class C>
__device__ __forceinline__ void fft_run(C* base, int es, const FftPlan& p, int i, bool active,
                                        const C* __restrict__ tw, int TN) {
  int Ns = 1;
  for (int s = 0; s < p.ns; ++s) {
    const int R = p.r[s];
    const int tstride = TN / (Ns * R);
    switch (R) {
      case 2:  if constexpr (E % 2 == 0)  fft_stage<2, E, S>(base, es, p.L, Ns, i, p.tpt, active, tw, tstride); break;
      case 3:  if constexpr (E % 3 == 0)  fft_stage<3, E, S>(base, es, p.L, Ns, i, p.tpt, active, tw, tstride); break;
      case 4:  if constexpr (E % 4 == 0)  fft_stage<4, E, S>(base, es, p.L, Ns, i, p.tpt, active, tw, tstride); break;
      case 5:  if constexpr (E % 5 == 0)  fft_stage<5, E, S>(base, es, p.L, Ns, i, p.tpt, active, tw, tstride); break;
      case 8:  if constexpr (E % 8 == 0)  fft_stage<8, E, S>(base, es, p.L, Ns, i, p.tpt, active, tw, tstride); break;
      case 16: if constexpr (E % 16 == 0) fft_stage<16, E, S>(base, es, p.L, Ns, i, p.tpt, active, tw, tstride); break;
      default: break;
    }
    Ns *= R;
  }
}

// Runs the plan on one transform per thread group.  Every thread of the block
// must call this (with active = false when it owns no transform), since each
// stage synchronizes the block.  The set of E values must match plan.cpp.
template <int S, class C>
__device__ __noinline__ void fft_smem(C* base, int es, const FftPlan& p, int i, bool active,
                                     const C* __restrict__ tw, int TN) {
  switch (p.E) {
    case 2:  fft_run<2, S>(base, es, p, i, active, tw, TN); break;
    case 3:  fft_run<3, S>(base, es, p, i, active, tw, TN); break;
    case 4:  fft_run<4, S>(base, es, p, i, active, tw, TN); break;
    case 5:  fft_run<5, S>(base, es, p, i, active, tw, TN); break;
    case 6:  fft_run<6, S>(base, es, p, i, active, tw, TN); break;
    case 8:  fft_run<8, S>(base, es, p, i, active, tw, TN); break;
    case 10: fft_run<10, S>(base, es, p, i, active, tw, TN); break;
    case 12: fft_run<12, S>(base, es, p, i, active, tw, TN); break;
    case 15: fft_run<15, S>(base, es, p, i, active, tw, TN); break;   // lengths with factors 3 and 5
    case 16: if constexpr (sizeof(C) == 8) fft_run<16, S>(base, es, p, i, active, tw, TN); break;
    case 20: if constexpr (sizeof(C) == 8) fft_run<20, S>(base, es, p, i, active, tw, TN); break;
    case 24: if constexpr (sizeof(C) == 8) fft_run<24, S>(base, es, p, i, active, tw, TN); break;
    case 30: if constexpr (sizeof(C) == 8) fft_run<30, S>(base, es, p, i, active, tw, TN); break;
    default: break;   // E = 1: length-1 transform, nothing to do
  }
}

}  // namespace dc

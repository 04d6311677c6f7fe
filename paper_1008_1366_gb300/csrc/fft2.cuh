// Sub-transform engine of the fused 1D kernels (conv1d.cuh).
//
// A length-L transform (L = product of the plan's radices) runs as Stockham
// stages: thread i of the tpt threads of a transform owns the butterflies
// j = i + b*tpt (b < E/R) of each radix-R stage; it gathers inputs
// x[j + q L/R], twiddles them by zeta_{Ns R}^{s q k} (k = j mod Ns, s = +1
// backward, -1 forward), applies the radix-R DFT and scatters to
// (j - k) R + k + q Ns.  Natural order in and out.  Plans put the powers of
// two first and the odd radices last, so every stage up to the first odd one
// starts at a power-of-two stride Ns (k is a mask there, a division after
// it); both directions use that order.
// The pointwise product is fused into the first forward stage (conv1d.cuh).
//
// Roots of unity come from two short tables in shared memory,
// zeta_TN^e = hi[e >> sh] * lo[e & mask], the factorization of Sec. 2.1 of
// the paper (one complex multiply per factor), filled from the FP64-generated
// table in global memory.
#pragma once

#include <type_traits>

#include "fft.cuh"

namespace dc {

template <class C> struct Roots {
  const C* lo;
  const C* hi;
  int sh, mask;
  __device__ __forceinline__ C at(int e) const { return cmul(hi[e >> sh], lo[e & mask]); }
};

// element idx of an array in shared memory: p[idx * es + (idx >> ps)]
// (contiguous and padded: es = 1, ps = 4 or 3; interleaved: es = w, ps = 31)
template <class C> struct Arr {
  C* p;
  int es, ps;
  __device__ __forceinline__ C& operator[](int idx) const { return p[idx * es + (idx >> ps)]; }
};

template <class C> __host__ __device__ constexpr int pad_shift() { return sizeof(C) == 8 ? 4 : 3; }
template <class C> __host__ __device__ constexpr int padded_len(int L) {
  return L + (L >> (sizeof(C) == 8 ? 4 : 3)) + 1;
}

// --- radix butterflies with a runtime sign s = +-1: y_k = sum_j x_j zeta_R^{s jk}

template <class C> __device__ __forceinline__ C si(C a, int s) {   // s * i * a
  C c;
  if (s > 0) { c.x = -a.y; c.y = a.x; } else { c.x = a.y; c.y = -a.x; }
  return c;
}
template <class C, class R> __device__ __forceinline__ C mcs(C a, R c, R sn, int s) {  // a (c + s i sn)
  C w; w.x = c; w.y = s > 0 ? sn : -sn; return cmul(a, w);
}
template <class C> __device__ __forceinline__ void r4(C& x0, C& x1, C& x2, C& x3, int s) {
  C t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3), t3 = si(csub(x1, x3), s);
  x0 = cadd(t0, t2); x2 = csub(t0, t2); x1 = cadd(t1, t3); x3 = csub(t1, t3);
}
template <class C> __device__ __forceinline__ void r8(C* x, int s) {
  using R = decltype(x[0].x);
  const R h = (R)0.70710678118654752440;
  r4(x[0], x[2], x[4], x[6], s);
  r4(x[1], x[3], x[5], x[7], s);
  C o1 = mcs(x[3], h, h, s), o2 = si(x[5], s), o3 = mcs(x[7], -h, h, s);
  C e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
  x[0] = cadd(e0, x[1]); x[4] = csub(e0, x[1]);
  x[1] = cadd(e1, o1);   x[5] = csub(e1, o1);
  x[2] = cadd(e2, o2);   x[6] = csub(e2, o2);
  x[3] = cadd(e3, o3);   x[7] = csub(e3, o3);
}
template <class C> __device__ __forceinline__ void r16(C* x, int s) {
  using R = decltype(x[0].x);
  C e[8], o[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) { e[j] = x[2 * j]; o[j] = x[2 * j + 1]; }
  r8(e, s);
  r8(o, s);
  const R c1 = (R)0.92387953251128675613, s1 = (R)0.38268343236508977173;  // cos, sin(pi/8)
  const R h = (R)0.70710678118654752440;
  o[1] = mcs(o[1], c1, s1, s); o[2] = mcs(o[2], h, h, s); o[3] = mcs(o[3], s1, c1, s);
  o[4] = si(o[4], s);
  o[5] = mcs(o[5], -s1, c1, s); o[6] = mcs(o[6], -h, h, s); o[7] = mcs(o[7], -c1, s1, s);
#pragma unroll
  for (int k = 0; k < 8; ++k) { x[k] = cadd(e[k], o[k]); x[k + 8] = csub(e[k], o[k]); }
}
template <class C> __device__ __forceinline__ void r3(C* x, int s) {
  using R = decltype(x[0].x);
  const R sn = (R)0.86602540378443864676;   // sin(2 pi / 3)
  C t = cadd(x[1], x[2]);
  C d = si(csub(x[1], x[2]), s);
  C a; a.x = x[0].x - (R)0.5 * t.x; a.y = x[0].y - (R)0.5 * t.y;
  x[0] = cadd(x[0], t);
  x[1].x = a.x + sn * d.x; x[1].y = a.y + sn * d.y;
  x[2].x = a.x - sn * d.x; x[2].y = a.y - sn * d.y;
}
template <class C> __device__ __forceinline__ void r5(C* x, int s) {
  using R = decltype(x[0].x);
  const R c1 = (R)0.30901699437494742410, c2 = (R)-0.80901699437494742410;  // cos(2pi/5), cos(4pi/5)
  const R s1 = (R)0.95105651629515357212, s2 = (R)0.58778525229247312917;   // sin(2pi/5), sin(4pi/5)
  C t1 = cadd(x[1], x[4]), t2 = cadd(x[2], x[3]), d1 = csub(x[1], x[4]), d2 = csub(x[2], x[3]);
  C a1, a2, u1, u2;
  a1.x = x[0].x + c1 * t1.x + c2 * t2.x; a1.y = x[0].y + c1 * t1.y + c2 * t2.y;
  a2.x = x[0].x + c2 * t1.x + c1 * t2.x; a2.y = x[0].y + c2 * t1.y + c1 * t2.y;
  u1.x = s1 * d1.x + s2 * d2.x; u1.y = s1 * d1.y + s2 * d2.y;
  u2.x = s2 * d1.x - s1 * d2.x; u2.y = s2 * d1.y - s1 * d2.y;
  C b1 = si(u1, s), b2 = si(u2, s);
  x[0] = cadd(x[0], cadd(t1, t2));
  x[1] = cadd(a1, b1); x[4] = csub(a1, b1);
  x[2] = cadd(a2, b2); x[3] = csub(a2, b2);
}
template <int R, class C> __device__ __forceinline__ void rdft(C* x, int s) {
  if constexpr (R == 2) { C t = x[0]; x[0] = cadd(t, x[1]); x[1] = csub(t, x[1]); }
  else if constexpr (R == 3) r3(x, s);
  else if constexpr (R == 4) r4(x[0], x[1], x[2], x[3], s);
  else if constexpr (R == 5) r5(x, s);
  else if constexpr (R == 8) r8(x, s);
  else if constexpr (R == 16) r16(x, s);
}

// twiddle + radix-R DFT for the NB butterflies a thread owns in one stage
template <int R, int NB, class C>
__device__ __forceinline__ void bfly(C* v, int i, int tpt, int Ns, int tstr, const Roots<C>& rt, int s) {
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    if (Ns > 1) {
      // Ns is a power of two up to the first odd radix (the odd radices come last)
      const int j = i + b * tpt;
      const int e = ((Ns & (Ns - 1)) ? j % Ns : j & (Ns - 1)) * tstr;
#pragma unroll
      for (int q = 1; q < R; ++q) {
        C w = rt.at(q * e);
        if (s < 0) w.y = -w.y;
        v[b * R + q] = cmul(v[b * R + q], w);
      }
    }
    rdft<R>(&v[b * R], s);
  }
}

// Invoke f with the compile-time radix of this stage (only radices that
// divide E are instantiated).
template <int E, class F> __device__ __forceinline__ void with_radix(int R, F&& f) {
  switch (R) {
    case 2:  if constexpr (E % 2 == 0)  f(std::integral_constant<int, 2>{}); break;
    case 3:  if constexpr (E % 3 == 0)  f(std::integral_constant<int, 3>{}); break;
    case 4:  if constexpr (E % 4 == 0)  f(std::integral_constant<int, 4>{}); break;
    case 5:  if constexpr (E % 5 == 0)  f(std::integral_constant<int, 5>{}); break;
    case 8:  if constexpr (E % 8 == 0)  f(std::integral_constant<int, 8>{}); break;
    case 16: if constexpr (E % 16 == 0) f(std::integral_constant<int, 16>{}); break;
    default: break;
  }
}

}  // namespace dc

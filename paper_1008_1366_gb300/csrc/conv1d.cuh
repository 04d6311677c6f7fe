// Fused implicitly dealiased 1D convolutions.
//
// For each residue r of the padded index (j = q l + r), one block:
//   1. builds the r-th sub-transform inputs from the unpadded data
//      (pre-twiddle by zeta_{qm}^{rk}, Eq. (2.1); centered/Hermitian w_{k,r},
//      Eqs. (2.4)-(2.5) and Sec. 2.3; ternary zeta_{4m}^{rk} U_k, Sec. 4.2),
//   2. runs the m-point backward sub-transforms,
//   3. forms the pointwise product,
//   4. runs the m-point forward sub-transform, and
//   5. accumulates zeta_{qm}^{-rk} times it into the output (Eq. (2.2),
//      Eqs. (2.6)/(2.7), Sec. 4.2); at the last residue the sum is scaled by
//      1/N and written.
// Steps 1-2 fuse the build into the first transform stage (loads straight
// from global memory), 2-4 meet in registers (fft2.cuh), and 4-5 fuse the
// recombination into the last stage, so each input is read once and each
// output written once.  The padded array of size qm never exists: per
// residue only m-point arrays live in shared memory (level 1) or, for m
// beyond shared memory, in a per-block scratch slot that the two-level
// decomposition m = L1 * L2 streams through in column and row tiles
// (level 2).
#pragma once

#include "fft2.cuh"
#include "plan.h"

namespace dc {

constexpr int kThreads = 512;

struct ConvArgs {
  const void* in[4];      // inputs (f, g, e), (w, f, g) for gradients, (f1, g1, f2, g2) for dot products
  void* out[2];           // outputs (h) or (df, dg)
  const int64_t* off;     // per-instance element offsets (device) or null: inst * stride
  int64_t stride;
  const int32_t* order;   // instance id of each item slot (device) or null: identity
  const Item* items;      // work items (device) or null: uniform items of cfg0.nt instances
  int32_t nitems;
  int32_t ninst;
  const CfgDev* cfgs;     // per-size configurations (device) or null: cfg0
  WorkHeader* hdr;
  char* scratch;          // level-2 scratch, slot_bytes per block
  int64_t slot_bytes;
  int32_t persistent;     // take items from hdr->counter
  int32_t pad;
  CfgDev cfg0;
};

template <class C> struct RealOf;
template <> struct RealOf<float2> { using type = float; };
template <> struct RealOf<double2> { using type = double; };

template <class C> struct Ctx {
  const C* in0;     // inputs and outputs as named pointers: never indexed at
  const C* in1;     // run time, so they stay in registers
  const C* in2;
  const C* in3;
  C* out0;
  C* out1;
  int m, TN;
  Roots<C> rt;
};

// input x of an instance (x = 0, 1, 2, 3)
template <class C> __device__ __forceinline__ const C* in_ptr(const Ctx<C>& c, int x) {
  return x == 0 ? c.in0 : (x == 1 ? c.in1 : (x == 2 ? c.in2 : c.in3));
}

// ---------------------------------------------------------------------------
// kind policies: residue inputs, pointwise product, recombination, scaling
// ---------------------------------------------------------------------------
template <int KIND, class C> struct KP;

// complex binary convolution, N = 2m, residues r = 0, 1 (Eqs. (2.1)-(2.2))
template <class C> struct KP<K_COMPLEX, C> {
  static constexpr int Q = 2, NARR = 2, NFWD = 1;
  __device__ static C build(const Ctx<C>& c, int x, int k, int ri, int m, const Roots<C>& rt) {
    C v = in_ptr(c, x)[k];
    return ri ? cmul(v, rt.at(k)) : v;
  }
  __device__ static void pointwise(C* v) { v[0] = cmul(v[0], v[1]); }
  __device__ static C contrib(int, C X, int k, int ri, int, const Roots<C>& rt) {
    return ri ? cmulc(X, rt.at(k)) : X;
  }
  __device__ static C finish(int, C a, int, int m) {
    using R = typename RealOf<C>::type;
    return cscale(a, (R)1 / (R)(2 * m));
  }
};

// w_{k,r} of the centered Hermitian transform (Sec. 2.3): U_0 at k = 0 (taken
// real: Hermitian symmetry enforced), else zeta_{3m}^{rk} (U_k + zeta_3^{-r}
// conj U_{m-k}); zeta_3^{-r} = (-1/2, -r sqrt(3)/2).  x0 overrides U_0.
template <class C>
__device__ __forceinline__ C herm_w(const C* u, int k, int r, int m, const Roots<C>& rt, C x0) {
  using R = typename RealOf<C>::type;
  if (k == 0) return x0;
  C a = u[k];
  C b = cconj(u[m - k]);
  if (r == 0) return cadd(a, b);
  C z3; z3.x = (R)-0.5; z3.y = (R)(-r) * (R)0.86602540378443864676;
  a = cadd(a, cmul(b, z3));
  C t = rt.at(k);
  return r > 0 ? cmul(a, t) : cmulc(a, t);
}

template <class C> __device__ __forceinline__ C pack_i(C a, C b) {  // a + i b
  C c; c.x = a.x - b.y; c.y = a.y + b.x; return c;
}

template <class C> __device__ __forceinline__ C herm_out_twiddle(C X, int k, int r, const Roots<C>& rt) {
  // zeta_{3m}^{-rk} X (Eq. (2.7))
  if (r == 0) return X;
  C t = rt.at(k);
  return r > 0 ? cmulc(X, t) : cmul(X, t);
}

template <class C> __device__ __forceinline__ C real_part(C a) { a.y = 0; return a; }

// centered Hermitian binary convolution, N = 3m, r = -1, 0, 1.  The two real
// backward transforms of f and g share one complex transform of
// w^f + i w^g (both results are real); the real product is forward
// transformed as a complex array with zero imaginary part.
template <class C> struct KP<K_HERMITIAN, C> {
  static constexpr int Q = 3, NARR = 1, NFWD = 1;
  __device__ static C build(const Ctx<C>& c, int, int k, int ri, int m, const Roots<C>& rt) {
    const int r = ri - 1;
    return pack_i(herm_w(c.in0, k, r, m, rt, real_part(c.in0[0])),
                  herm_w(c.in1, k, r, m, rt, real_part(c.in1[0])));
  }
  __device__ static void pointwise(C* v) { v[0].x = v[0].x * v[0].y; v[0].y = 0; }
  __device__ static C contrib(int, C X, int k, int ri, int, const Roots<C>& rt) {
    return herm_out_twiddle(X, k, ri - 1, rt);
  }
  __device__ static C finish(int, C a, int, int m) {
    using R = typename RealOf<C>::type;
    return cscale(a, (R)1 / (R)(3 * m));
  }
};

// V_k of the ternary transform (Sec. 4.2): zeta_{4m}^{rk} U_k for k < m (U_0
// real), 0 at k = m, conj(V_{2m-k}) for m < k < 2m.
template <class C>
__device__ __forceinline__ C tern_v(const C* u, int k, int r, int m, const Roots<C>& rt) {
  if (k == m) { C z; z.x = 0; z.y = 0; return z; }
  const bool up = k > m;
  const int kk = up ? 2 * m - k : k;
  C x = u[kk];
  if (kk == 0) x.y = 0;
  if (r) x = cmul(x, rt.at(kk));
  return up ? cconj(x) : x;
}

// centered Hermitian ternary convolution, N = 4m, r = 0, 1, sub-transforms of
// length 2m: (V^f + i V^g) and V^e backward, the triple real product forward.
template <class C> struct KP<K_TERNARY, C> {
  static constexpr int Q = 2, NARR = 2, NFWD = 1;
  __device__ static C build(const Ctx<C>& c, int x, int k, int ri, int m, const Roots<C>& rt) {
    if (x == 0) return pack_i(tern_v(c.in0, k, ri, m, rt), tern_v(c.in1, k, ri, m, rt));
    return tern_v(c.in2, k, ri, m, rt);
  }
  __device__ static void pointwise(C* v) { v[0].x = v[0].x * v[0].y * v[1].x; v[0].y = 0; }
  __device__ static C contrib(int, C X, int k, int ri, int, const Roots<C>& rt) {
    return ri ? cmulc(X, rt.at(k)) : X;
  }
  __device__ static C finish(int, C a, int, int m) {
    using R = typename RealOf<C>::type;
    return cscale(a, (R)1 / (R)(4 * m));
  }
};

// gradient of the complex convolution: inputs (w, f, g); the residue
// transforms of w, f, g are shared and the products W conj(G) -> df,
// W conj(F) -> dg are forward transformed (N = 2m correlation).
template <class C> struct KP<K_COMPLEX_ADJ, C> {
  static constexpr int Q = 2, NARR = 3, NFWD = 2;
  __device__ static C build(const Ctx<C>& c, int x, int k, int ri, int m, const Roots<C>& rt) {
    return KP<K_COMPLEX, C>::build(c, x, k, ri, m, rt);
  }
  __device__ static void pointwise(C* v) {
    C a = cmulc(v[0], v[2]);
    C b = cmulc(v[0], v[1]);
    v[0] = a; v[1] = b;
  }
  __device__ static C contrib(int o, C X, int k, int ri, int m, const Roots<C>& rt) {
    return KP<K_COMPLEX, C>::contrib(o, X, k, ri, m, rt);
  }
  __device__ static C finish(int o, C a, int k, int m) { return KP<K_COMPLEX, C>::finish(o, a, k, m); }
};

// gradient of the Hermitian convolution: inputs (w, f, g).  W = w with
// W_0 = 2 Re w_0; df = S conv(W, g), dg = S conv(W, f) with S = 1/2 at k = 0.
// W is transformed alone (so the result is exactly linear in w); f and g
// share the second transform; the two real products are forward transformed.
template <class C> struct KP<K_HERMITIAN_ADJ, C> {
  static constexpr int Q = 3, NARR = 2, NFWD = 2;
  __device__ static C build(const Ctx<C>& c, int x, int k, int ri, int m, const Roots<C>& rt) {
    const int r = ri - 1;
    if (x == 0) {
      C w0 = real_part(c.in0[0]);
      w0.x *= 2;
      return herm_w(c.in0, k, r, m, rt, w0);
    }
    return pack_i(herm_w(c.in1, k, r, m, rt, real_part(c.in1[0])),
                  herm_w(c.in2, k, r, m, rt, real_part(c.in2[0])));
  }
  __device__ static void pointwise(C* v) {
    const auto uw = v[0].x, uf = v[1].x, ug = v[1].y;
    v[0].x = uw * ug; v[0].y = 0;
    v[1].x = uw * uf; v[1].y = 0;
  }
  __device__ static C contrib(int, C X, int k, int ri, int, const Roots<C>& rt) {
    return herm_out_twiddle(X, k, ri - 1, rt);
  }
  __device__ static C finish(int, C a, int k, int m) {
    using R = typename RealOf<C>::type;
    R s = (R)1 / (R)(3 * m);
    if (k == 0) s *= (R)0.5;
    return cscale(a, s);
  }
};

// rows of the multi-D Hermitian gradient: two plain Hermitian convolutions
// (W, g) -> out 0 and (W, f) -> out 1 sharing the transforms of W; the
// symmetrization of W and the halving act on the whole multi-D array and are
// done by the outer passes.
template <class C> struct KP<K_HERMITIAN_PAIR, C> {
  static constexpr int Q = 3, NARR = 2, NFWD = 2;
  __device__ static C build(const Ctx<C>& c, int x, int k, int ri, int m, const Roots<C>& rt) {
    const int r = ri - 1;
    if (x == 0) return herm_w(c.in0, k, r, m, rt, real_part(c.in0[0]));
    return pack_i(herm_w(c.in1, k, r, m, rt, real_part(c.in1[0])),
                  herm_w(c.in2, k, r, m, rt, real_part(c.in2[0])));
  }
  __device__ static void pointwise(C* v) { KP<K_HERMITIAN_ADJ, C>::pointwise(v); }
  __device__ static C contrib(int o, C X, int k, int ri, int m, const Roots<C>& rt) {
    return KP<K_HERMITIAN_ADJ, C>::contrib(o, X, k, ri, m, rt);
  }
  __device__ static C finish(int o, C a, int k, int m) { return KP<K_HERMITIAN, C>::finish(o, a, k, m); }
};

// Inputs as arrays of vectors (Sec. 3, 2D pseudospectral application): the
// product f * g read as the dot product f1 * g1 + f2 * g2 of two pairs.  The
// four inputs take one backward transform each per residue (Eq. (2.1)); the
// two pointwise products are summed in physical space, so one forward
// transform per residue (Eq. (2.2)) serves both pairs: five transforms per
// residue instead of six.
template <class C> struct KP<K_COMPLEX_DOT2, C> {
  static constexpr int Q = 2, NARR = 4, NFWD = 1;
  __device__ static C build(const Ctx<C>& c, int x, int k, int ri, int m, const Roots<C>& rt) {
    return KP<K_COMPLEX, C>::build(c, x, k, ri, m, rt);
  }
  __device__ static void pointwise(C* v) { v[0] = cadd(cmul(v[0], v[1]), cmul(v[2], v[3])); }
  __device__ static C contrib(int o, C X, int k, int ri, int m, const Roots<C>& rt) {
    return KP<K_COMPLEX, C>::contrib(o, X, k, ri, m, rt);
  }
  __device__ static C finish(int o, C a, int k, int m) { return KP<K_COMPLEX, C>::finish(o, a, k, m); }
};

// The centered Hermitian dot product of two pairs (same passage, Sec. 2.3):
// each pair's real backward transforms share one complex transform of
// w^f + i w^g, so the two real products need two backward transforms and
// their sum one forward transform per residue (three, against four for two
// separate convolutions).
template <class C> struct KP<K_HERMITIAN_DOT2, C> {
  static constexpr int Q = 3, NARR = 2, NFWD = 1;
  __device__ static C build(const Ctx<C>& c, int x, int k, int ri, int m, const Roots<C>& rt) {
    const int r = ri - 1;
    const C* a = x ? c.in2 : c.in0;
    const C* b = x ? c.in3 : c.in1;
    return pack_i(herm_w(a, k, r, m, rt, real_part(a[0])), herm_w(b, k, r, m, rt, real_part(b[0])));
  }
  __device__ static void pointwise(C* v) {
    v[0].x = v[0].x * v[0].y + v[1].x * v[1].y;
    v[0].y = 0;
  }
  __device__ static C contrib(int o, C X, int k, int ri, int m, const Roots<C>& rt) {
    return KP<K_HERMITIAN, C>::contrib(o, X, k, ri, m, rt);
  }
  __device__ static C finish(int o, C a, int k, int m) { return KP<K_HERMITIAN, C>::finish(o, a, k, m); }
};

// ---------------------------------------------------------------------------
// stage interpreter.  Every transform stage of every path is one call of
// stage_call (or boundary_call for the stage that meets the product), with
// its source and destination described at run time:
//   sources:      SMEM   shared-memory array
//                 BUILD  residue input of the kind, element k = kb + idx*ks
//                 GLOBAL scratch g[gb + idx*gs]
//   destinations: SMEM   shared-memory array
//                 GTW    scratch g[gb + idx*gs] = v * zeta_TN^{+-idx*twm}
//                 SINK   recombination into output o at k = kb + idx*ks
//                        (accumulator h[idx], thread-private across residues)
// One compiled copy per (kind, precision, E) keeps the code, and the build,
// small.
// ---------------------------------------------------------------------------
enum : int { SRC_SMEM = 0, SRC_BUILD = 1, SRC_GLOBAL = 2 };
enum : int { DST_SMEM = 0, DST_GTW = 1, DST_SINK = 2 };

template <class C> struct Src {
  int mode, x, ri, kb, ks, gs;
  Arr<C> a;
  const C* g;
  int64_t gb;
};
template <class C> struct Dst {
  int mode, o, ri, kb, ks, gs, twm, tsgn;
  Arr<C> a, h;
  C* g;
  int64_t gb;
};
template <class C> __device__ __forceinline__ Src<C> src_smem(Arr<C> a) {
  Src<C> s{}; s.mode = SRC_SMEM; s.a = a; return s;
}
template <class C> __device__ __forceinline__ Src<C> src_build(int x, int ri, int kb, int ks) {
  Src<C> s{}; s.mode = SRC_BUILD; s.x = x; s.ri = ri; s.kb = kb; s.ks = ks; return s;
}
template <class C> __device__ __forceinline__ Src<C> src_global(const C* g, int64_t gb, int gs) {
  Src<C> s{}; s.mode = SRC_GLOBAL; s.g = g; s.gb = gb; s.gs = gs; return s;
}
template <class C> __device__ __forceinline__ Dst<C> dst_smem(Arr<C> a) {
  Dst<C> d{}; d.mode = DST_SMEM; d.a = a; return d;
}
template <class C> __device__ __forceinline__ Dst<C> dst_gtw(C* g, int64_t gb, int gs, int twm, int tsgn) {
  Dst<C> d{}; d.mode = DST_GTW; d.g = g; d.gb = gb; d.gs = gs; d.twm = twm; d.tsgn = tsgn; return d;
}
template <class C> __device__ __forceinline__ Dst<C> dst_sink(int o, int ri, int kb, int ks, Arr<C> h) {
  Dst<C> d{}; d.mode = DST_SINK; d.o = o; d.ri = ri; d.kb = kb; d.ks = ks; d.h = h; return d;
}

template <int KIND, class C>
__device__ __forceinline__ C load_src(const Src<C>& s, const Ctx<C>& c, int idx) {
  if (s.mode == SRC_SMEM) return s.a[idx];
  if (s.mode == SRC_BUILD) return KP<KIND, C>::build(c, s.x, s.kb + idx * s.ks, s.ri, c.m, c.rt);
  return s.g[s.gb + (int64_t)idx * s.gs];
}

template <int KIND, class C>
__device__ __forceinline__ void store_dst(const Dst<C>& d, const Ctx<C>& c, int idx, C v) {
  using K = KP<KIND, C>;
  if (d.mode == DST_SMEM) {
    d.a[idx] = v;
  } else if (d.mode == DST_GTW) {
    C w = c.rt.at(idx * d.twm);
    d.g[d.gb + (int64_t)idx * d.gs] = d.tsgn > 0 ? cmul(v, w) : cmulc(v, w);
  } else {
    const int k = d.kb + idx * d.ks;
    if (k < c.m) {
      const C cv = K::contrib(d.o, v, k, d.ri, c.m, c.rt);
      if (d.ri == 0) d.h[idx] = cv;
      else if (d.ri < K::Q - 1) d.h[idx] = cadd(d.h[idx], cv);
      else (d.o == 0 ? c.out0 : c.out1)[k] = K::finish(d.o, cadd(d.h[idx], cv), k, c.m);
    }
  }
}

// one Stockham stage of radix RR: gather x[j + q L/RR] from src, twiddle +
// DFT, scatter to (j - k) RR + k + q Ns in dst.  sync_mid: barrier between
// gather and scatter (in-place shared-memory stages).  Plain parameters and
// an explicit radix switch (no capturing lambdas) keep every local in
// registers.
template <int RR, int E, int KIND, int SM, int DM, class C>
__device__ __forceinline__ void stage_r(int Ns, int L, int tpt, int sgn, Src<C> src, Dst<C> dst,
                                        bool sync_mid, int i, bool act, const Ctx<C>& ctx) {
  constexpr int NB = E / RR;
  using K = KP<KIND, C>;
  C v[E];
  // the source / destination switch sits outside the unrolled loops
  if (act) {
    const int LR = L / RR;
    if constexpr (SM == SRC_SMEM) {
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int q = 0; q < RR; ++q) v[b * RR + q] = src.a[i + b * tpt + q * LR];
    } else if constexpr (SM == SRC_BUILD) {
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int q = 0; q < RR; ++q)
          v[b * RR + q] = K::build(ctx, src.x, src.kb + (i + b * tpt + q * LR) * src.ks, src.ri,
                                   ctx.m, ctx.rt);
    } else {
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int q = 0; q < RR; ++q)
          v[b * RR + q] = src.g[src.gb + (int64_t)(i + b * tpt + q * LR) * src.gs];
    }
  }
  if (sync_mid) __syncthreads();
  if (act) {
    bfly<RR, NB>(v, i, tpt, Ns, ctx.TN / (Ns * RR), ctx.rt, sgn);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = i + b * tpt;
      // Ns is a power of two up to the first odd radix (the odd radices come last)
      const int k = (Ns & (Ns - 1)) ? j % Ns : j & (Ns - 1);
      const int ob = (j - k) * RR + k;
#pragma unroll
      for (int q = 0; q < RR; ++q) {
        const int idx = ob + q * Ns;
        if constexpr (DM == DST_SMEM) {
          dst.a[idx] = v[b * RR + q];
        } else if constexpr (DM == DST_GTW) {
          const C w = ctx.rt.at(idx * dst.twm);
          dst.g[dst.gb + (int64_t)idx * dst.gs] = dst.tsgn > 0 ? cmul(v[b * RR + q], w) : cmulc(v[b * RR + q], w);
        } else {
          store_dst<KIND>(dst, ctx, idx, v[b * RR + q]);
        }
      }
    }
  }
}

template <int E, int KIND, int SM, int DM, class C>
__device__ __forceinline__ void stage_body(int R, int Ns, int L, int tpt, int sgn, Src<C> src,
                                           Dst<C> dst, bool sync_mid, int i, bool act,
                                           const Ctx<C>& ctx) {
  switch (R) {
#define DC_STAGE_CASE(RV)                                                                              \
    case RV:                                                                                           \
      if constexpr (E % RV == 0) stage_r<RV, E, KIND, SM, DM>(Ns, L, tpt, sgn, src, dst, sync_mid, i, act, ctx); \
      break;
    DC_STAGE_CASE(2)
    DC_STAGE_CASE(3)
    DC_STAGE_CASE(4)
    DC_STAGE_CASE(5)
    DC_STAGE_CASE(8)
    DC_STAGE_CASE(16)
#undef DC_STAGE_CASE
    default: break;
  }
}

// The product stage: after the last backward stage (an ordinary in-place
// stage) every thread gathers, at the inputs of its first forward
// butterflies, the values of all arrays, forms the pointwise product on the
// fly (only the NFWD products stay live), applies the first forward stage
// (Ns = 1, no twiddles) and writes back in place.  Arrays A[x] = base +
// x * astride, padded layout.
template <int RR, int E, int KIND, class C>
__device__ __forceinline__ void product_r(int L, int tpt, C* base, int astride, int i, bool act,
                                          const Ctx<C>& ctx) {
  using K = KP<KIND, C>;
  constexpr int PS = pad_shift<C>();
  constexpr int NB = E / RR;
  C v[K::NFWD][E];
  if (act) {
    const int LR = L / RR;
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int q = 0; q < RR; ++q) {
        const int idx = i + b * tpt + q * LR;
        C w[K::NARR];
#pragma unroll
        for (int x = 0; x < K::NARR; ++x) w[x] = base[x * astride + idx + (idx >> PS)];
        K::pointwise(w);
#pragma unroll
        for (int o = 0; o < K::NFWD; ++o) v[o][b * RR + q] = w[o];
      }
  }
  __syncthreads();
  if (act) {
#pragma unroll
    for (int o = 0; o < K::NFWD; ++o) {
      bfly<RR, NB>(v[o], i, tpt, 1, 1, ctx.rt, -1);
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int q = 0; q < RR; ++q) {
          const int idx = (i + b * tpt) * RR + q;
          base[o * astride + idx + (idx >> PS)] = v[o][b * RR + q];
        }
    }
  }
}

template <int E, int KIND, class C>
__device__ __forceinline__ void product_body(int R, int L, int tpt, C* base, int astride, int i, bool act,
                                             const Ctx<C>& ctx) {
  switch (R) {
#define DC_PROD_CASE(RV)                                                                   \
    case RV:                                                                               \
      if constexpr (E % RV == 0) product_r<RV, E, KIND>(L, tpt, base, astride, i, act, ctx); \
      break;
    DC_PROD_CASE(2)
    DC_PROD_CASE(3)
    DC_PROD_CASE(4)
    DC_PROD_CASE(5)
    DC_PROD_CASE(8)
    DC_PROD_CASE(16)
#undef DC_PROD_CASE
    default: break;
  }
}

// A phase of an item, from the thread's point of view:
//   PH_L1  one residue of a level-1 convolution on this thread's instance
//   PH_A   pass A: backward column transform of array x, residue ri, at k1
//   PH_B   pass B: one residue of the row convolution of row j2
//   PH_C   pass C: forward column transform of output x, residue ri, at k1
// Shared arrays: L1/B: A[x] = base + x * astride (padded); A/C: the column
// tile at base (interleaved, stride w); pass C accumulators at hbase.
enum : int { PH_L1 = 0, PH_A = 1, PH_B = 2, PH_C = 3 };
template <class C> struct Phase {
  int type, ri, x, i, aux, astride;
  bool act;
  C* base;
  C* hbase;
  const FftPlan* p;   // in shared memory
};

template <int KIND, class C>
__device__ __forceinline__ Src<C> phase_src0(const Phase<C>& P, const CfgDev& cfg, C* scr, int x) {
  using K = KP<KIND, C>;
  switch (P.type) {
    case PH_L1: return src_build<C>(x, P.ri, 0, 1);
    case PH_A:  return src_build<C>(P.x, P.ri, P.aux, cfg.L1);
    case PH_B:  return src_global<C>(scr + (size_t)(P.ri * K::NARR + x) * cfg.L, (int64_t)P.aux * cfg.L1, 1);
    default:    return src_global<C>(scr + (size_t)(P.ri * K::NARR + P.x) * cfg.L, P.aux, cfg.L1);
  }
}

template <int KIND, class C>
__device__ __forceinline__ Dst<C> phase_dstN(const Phase<C>& P, const CfgDev& cfg, C* scr, int o) {
  using K = KP<KIND, C>;
  constexpr int PS = pad_shift<C>();
  const int tq = cfg.TN / cfg.L;
  switch (P.type) {
    case PH_L1:
      return dst_sink<C>(o, P.ri, 0, 1, Arr<C>{P.base + K::NARR * P.astride + o * padded_len<C>(cfg.m), 1, PS});
    case PH_A:
      return dst_gtw<C>(scr + (size_t)(P.ri * K::NARR + P.x) * cfg.L, P.aux, cfg.L1, P.aux * tq, 1);
    case PH_B:
      return dst_gtw<C>(scr + (size_t)(P.ri * K::NARR + o) * cfg.L, (int64_t)P.aux * cfg.L1, 1, P.aux * tq, -1);
    default:
      return dst_sink<C>(P.x, P.ri, P.aux, cfg.L1, Arr<C>{P.hbase, cfg.w, 31});
  }
}

// Runs a phase as a flat sequence of stage operations; this loop holds the
// only copy of the stage code and of the product code for its E.
template <int E, int KIND, class C>
__device__ __forceinline__ void run_phase(const Phase<C>& P, const CfgDev& cfg, C* scr, const Ctx<C>& ctx) {
  using K = KP<KIND, C>;
  constexpr int PS = pad_shift<C>();
  const FftPlan& p = *P.p;
  const int ns = p.ns, L = p.L, tpt = p.tpt;
  const bool one = P.type == PH_A || P.type == PH_C;
  const bool fwd = P.type == PH_C;
  const int nb = K::NARR * ns;
  const int nops = one ? ns : nb + 1 + K::NFWD * (ns - 1);
  for (int op = 0; op < nops; ++op) {
    int R, Ns = 1, sgn = 1, arr = 0, s;
    bool sync_mid = true, sync_after = true, first, last;
    if (one) {
      s = op;
      R = p.r[s];
      for (int t = 0; t < s; ++t) Ns *= p.r[t];
      first = s == 0;
      last = s == ns - 1;
      sgn = fwd ? -1 : 1;
    } else if (op < nb) {             // backward stages, stage-major: stage s of every array
      s = op / K::NARR;
      arr = op % K::NARR;
      R = p.r[s];
      for (int t = 0; t < s; ++t) Ns *= p.r[t];
      first = s == 0;
      last = false;
      // first stages read global memory: one barrier after the last array
      sync_mid = s > 0;
      sync_after = s > 0 || arr == K::NARR - 1;
    } else if (op == nb) {            // product + first forward stage
      product_body<E, KIND>(p.r[0], L, tpt, P.base, P.astride, P.i, P.act, ctx);
      __syncthreads();
      continue;
    } else {                          // forward stages 1.. of output arr (same radix order)
      const int o = op - nb - 1;
      arr = o / (ns - 1);
      s = o % (ns - 1) + 1;
      R = p.r[s];
      for (int t = 0; t < s; ++t) Ns *= p.r[t];
      first = false;
      last = s == ns - 1;
      sync_mid = !last;
      sync_after = !last || arr == K::NFWD - 1;
      sgn = -1;
    }
    const Arr<C> a = one ? Arr<C>{P.base, cfg.w, 31} : Arr<C>{P.base + arr * P.astride, 1, PS};
    const Src<C> src = first ? phase_src0<KIND>(P, cfg, scr, arr) : src_smem(a);
    const Dst<C> dst = last ? phase_dstN<KIND>(P, cfg, scr, arr) : dst_smem(a);
    // one compiled stage per (source, destination) pair that occurs
    const int sm_ = src.mode, dm_ = dst.mode;
    if (sm_ == SRC_SMEM && dm_ == DST_SMEM)
      stage_body<E, KIND, SRC_SMEM, DST_SMEM>(R, Ns, L, tpt, sgn, src, dst, sync_mid, P.i, P.act, ctx);
    else if (sm_ == SRC_BUILD)
      stage_body<E, KIND, SRC_BUILD, DST_SMEM>(R, Ns, L, tpt, sgn, src, dst, sync_mid, P.i, P.act, ctx);
    else if (sm_ == SRC_GLOBAL)
      stage_body<E, KIND, SRC_GLOBAL, DST_SMEM>(R, Ns, L, tpt, sgn, src, dst, sync_mid, P.i, P.act, ctx);
    else if (dm_ == DST_SINK)
      stage_body<E, KIND, SRC_SMEM, DST_SINK>(R, Ns, L, tpt, sgn, src, dst, sync_mid, P.i, P.act, ctx);
    else
      stage_body<E, KIND, SRC_SMEM, DST_GTW>(R, Ns, L, tpt, sgn, src, dst, sync_mid, P.i, P.act, ctx);
    if (sync_after) __syncthreads();
  }
}

template <class C> __device__ __forceinline__ Ctx<C> inst_ctx(const ConvArgs& a, int slot, int m, int TN,
                                                             const Roots<C>& rt) {
  Ctx<C> c{};
  const int inst = a.order ? a.order[slot] : slot;
  const int64_t off = a.off ? a.off[inst] : (int64_t)inst * a.stride;
  c.in0 = a.in[0] ? (const C*)a.in[0] + off : nullptr;
  c.in1 = a.in[1] ? (const C*)a.in[1] + off : nullptr;
  c.in2 = a.in[2] ? (const C*)a.in[2] + off : nullptr;
  c.in3 = a.in[3] ? (const C*)a.in[3] + off : nullptr;
  c.out0 = a.out[0] ? (C*)a.out[0] + off : nullptr;
  c.out1 = a.out[1] ? (C*)a.out[1] + off : nullptr;
  c.m = m;
  c.TN = TN;
  c.rt = rt;
  return c;
}

// tiny transforms (L not a multiple of the plan's E): the DFTs by definition,
// one thread per element
template <int KIND, class C>
__device__ void conv_level1_direct(const ConvArgs& a, const CfgDev& cfg, int first, int count, C* sm,
                                   const Roots<C>& rt) {
  using K = KP<KIND, C>;
  const int L = cfg.L, m = cfg.m, step = cfg.TN / L;
  const int t = threadIdx.x / L, i = threadIdx.x - t * L;
  const bool act = t < count;
  Ctx<C> ctx{};
  if (act) ctx = inst_ctx<C>(a, first + t, m, cfg.TN, rt);
  ctx.m = m; ctx.TN = cfg.TN; ctx.rt = rt;
  C* base = sm + (size_t)(act ? t : 0) * (K::NARR * L + K::NFWD * m);
  for (int ri = 0; ri < K::Q; ++ri) {
    if (act)
      for (int x = 0; x < K::NARR; ++x) base[x * L + i] = K::build(ctx, x, i, ri, m, rt);
    __syncthreads();
    C v[K::NARR];
    if (act) {
      for (int x = 0; x < K::NARR; ++x) {
        C s; s.x = 0; s.y = 0;
        for (int k = 0; k < L; ++k) s = cadd(s, cmul(base[x * L + k], rt.at(((i * k) % L) * step)));
        v[x] = s;
      }
      K::pointwise(v);
    }
    __syncthreads();
    if (act)
      for (int o = 0; o < K::NFWD; ++o) base[o * L + i] = v[o];
    __syncthreads();
    if (act) {
      for (int o = 0; o < K::NFWD; ++o) {
        C s; s.x = 0; s.y = 0;
        for (int j = 0; j < L; ++j) s = cadd(s, cmulc(base[o * L + j], rt.at(((i * j) % L) * step)));
        const Dst<C> d = dst_sink<C>(o, ri, 0, 1, Arr<C>{base + K::NARR * L + o * m, 1, 31});
        store_dst<KIND>(d, ctx, i, s);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Phases of an item.
// level 1 (count instances wholly in shared memory): one CONV phase per
//   residue: build -> transforms -> product -> transform -> recombination.
// level 2 (one instance, L = L1 * L2 through a scratch slot).  Backward DFT
//   of length L with k = k1 + L1 k2, j = j2 + L2 j1:
//   pass A (column tiles, ONE phases): X[k1][j2] = sum_{k2} zeta_{L2}^{j2 k2}
//            U[k1 + L1 k2], times zeta_L^{j2 k1}, stored row-major S[j2][k1];
//   pass B (row tiles, CONV phases): u[j2 + L2 j1] = sum_{k1} zeta_{L1}^{j1 k1}
//            S[j2][k1]; pointwise product; the forward transform runs the same
//            steps in reverse: length-L1 forward DFT over j1, times
//            zeta_L^{-j2 k1};
//   pass C (column tiles, ONE phases): length-L2 forward DFT over j2, then the
//            residue recombination into the output tile.
// The scrambled order between the halves is never undone (Sec. 1 notes bit
// reversal is unnecessary for a convolution).
// ---------------------------------------------------------------------------
template <int KIND, class C>
__device__ __forceinline__ int phase_count(const CfgDev& cfg) {
  using K = KP<KIND, C>;
  if (cfg.level == 1) return K::Q;
  const int ta = cfg.L1 / cfg.w, tb = cfg.L2 / cfg.nr;
  return ta * K::Q * K::NARR + tb * K::Q + ta * K::Q * K::NFWD;
}

template <class C> __host__ __device__ inline int roots_shift(int TN) {
  int lg = 0;
  while ((1 << lg) < TN) ++lg;
  return (lg + 1) / 2;
}
// shared-memory entries the two root tables of a size need
template <class C> __host__ __device__ inline int roots_entries(int TN) {
  const int sh = roots_shift<C>(TN);
  return (1 << sh) + ((TN + (1 << sh) - 1) >> sh) + 2;
}

template <int KIND, class C, class F> __device__ __forceinline__ void by_e(int E, F&& f) {
  if constexpr (sizeof(C) == 8) {
    if (E == 16) f(std::integral_constant<int, 16>{});
    else if (E == 12) f(std::integral_constant<int, 12>{});
    else if (E == 20) f(std::integral_constant<int, 20>{});
  } else {
    if (E == 8) f(std::integral_constant<int, 8>{});
    else if (E == 12) f(std::integral_constant<int, 12>{});
    else if (E == 10) f(std::integral_constant<int, 10>{});
  }
}

template <int KIND, class C>
__device__ __forceinline__ Phase<C> make_phase(const CfgDev& cfg, int ph, int count, C* sm) {
  using K = KP<KIND, C>;
  Phase<C> P{};
  if (cfg.level == 1) {
    const int tpt = cfg.p.tpt, t = threadIdx.x / tpt;
    P.type = PH_L1;
    P.ri = ph;
    P.p = &cfg.p;
    P.i = threadIdx.x - t * tpt;
    P.act = t < count;
    P.astride = padded_len<C>(cfg.L);
    P.base = sm + (size_t)(P.act ? t : 0) * (K::NARR * P.astride + K::NFWD * padded_len<C>(cfg.m));
    return P;
  }
  const int L1 = cfg.L1, L2 = cfg.L2, w = cfg.w, nr = cfg.nr;
  const int ta = L1 / w, tb = L2 / nr;
  const int na = ta * K::Q * K::NARR, nb = tb * K::Q;
  if (ph < na || ph >= na + nb) {
    const bool a = ph < na;
    int r = a ? ph : ph - na - nb;
    const int per_res = a ? K::NARR : K::NFWD;
    const int tile = r / (K::Q * per_res);
    r %= K::Q * per_res;
    const int c = threadIdx.x % w;
    P.type = a ? PH_A : PH_C;
    P.ri = r / per_res;
    P.x = r % per_res;
    P.aux = tile * w + c;
    P.p = &cfg.pc;
    P.i = threadIdx.x / w;
    P.act = P.i < cfg.pc.tpt;
    P.base = sm + c;
    P.hbase = sm + (size_t)(1 + P.x) * w * L2 + c;
    return P;
  }
  const int r = ph - na;
  const int rr = threadIdx.x / cfg.pr.tpt;
  P.type = PH_B;
  P.ri = r % K::Q;
  P.p = &cfg.pr;
  P.i = threadIdx.x - rr * cfg.pr.tpt;
  P.act = rr < nr;
  P.aux = (r / K::Q) * nr + (P.act ? rr : 0);
  P.astride = nr * padded_len<C>(L1);
  P.base = sm + (size_t)(P.act ? rr : 0) * padded_len<C>(L1);
  return P;
}

template <int KIND, class C>
__device__ __forceinline__ void run_item(const ConvArgs& a, const CfgDev& cfg, int first, int count, C* sm,
                                         const Roots<C>& rt) {
  if (cfg.level == 1 && cfg.p.E == 0) {
    conv_level1_direct<KIND, C>(a, cfg, first, count, sm, rt);
    return;
  }
  C* scr = (C*)(a.scratch + (size_t)blockIdx.x * a.slot_bytes);
  Ctx<C> ctx{};
  if (cfg.level == 2) {
    ctx = inst_ctx<C>(a, first, cfg.m, cfg.TN, rt);
  } else {
    const int t = threadIdx.x / cfg.p.tpt;
    ctx = inst_ctx<C>(a, first + (t < count ? t : 0), cfg.m, cfg.TN, rt);
  }
  const int nph = phase_count<KIND, C>(cfg);
  for (int ph = 0; ph < nph; ++ph) {
    const Phase<C> P = make_phase<KIND, C>(cfg, ph, count, sm);
    by_e<KIND, C>(P.p->E, [&](auto e) { run_phase<decltype(e)::value, KIND, C>(P, cfg, scr, ctx); });
  }
}

template <int KIND, class C>
__global__ void __launch_bounds__(kThreads, 1) conv1d_kernel(ConvArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ CfgDev s_cfg;
  __shared__ int s_item[3];
  int it = blockIdx.x;
  int cur_tn = -1;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      if (a.persistent) it = (int)atomicAdd(&a.hdr->counter, 1u);
      int cfgi = 0, first = 0, count = 0;
      if (it < a.nitems) {
        if (a.items) {
          const Item im = a.items[it];
          cfgi = im.cfg; first = im.first; count = im.count;
        } else {
          first = it * a.cfg0.nt;
          count = min(a.cfg0.nt, a.ninst - first);
        }
        s_cfg = a.cfgs ? a.cfgs[cfgi] : a.cfg0;
      }
      s_item[0] = it; s_item[1] = first; s_item[2] = count;
    }
    __syncthreads();
    it = s_item[0];
    if (it >= a.nitems) break;
    // the two root tables for this size, at the front of dynamic shared memory
    C* rt_mem = reinterpret_cast<C*>(smem_raw);
    const int TN = s_cfg.TN;
    const int sh = roots_shift<C>(TN), S = 1 << sh, nhi = (TN + S - 1) >> sh;
    if (TN != cur_tn) {
      const C* tw = (const C*)s_cfg.tw;
      for (int e = threadIdx.x; e < S + nhi; e += blockDim.x)
        rt_mem[e] = e < S ? tw[e < TN ? e : 0] : tw[(e - S) << sh];
      cur_tn = TN;
      __syncthreads();
    }
    const Roots<C> rt{rt_mem, rt_mem + S, sh, S - 1};
    C* sm = rt_mem + ((roots_entries<C>(TN) + 1) & ~1);
    run_item<KIND, C>(a, s_cfg, s_item[1], s_item[2], sm, rt);
    if (!a.persistent) it += gridDim.x;
  }
}

}  // namespace dc

// Fixed-shape engine: implicitly dealiased convolutions (FP32 and FP64
// builds) whose sizes are known at compile time.
//
// Every size m of the set {2^a, 3*2^a, 5*2^a} in [64, 65536] gets its own
// code: radices, threads per transform, tile shapes and every shared-memory
// index are compile-time constants, so stages are straight-line code with
// immediate offsets (a runtime-shaped stage loop keeps its descriptors live
// across the loop and spills).
//
// Method (Sec. 2.1 of the paper): with N = 2m and residues r = 0, 1,
//   u_{2l+r} = sum_k zeta_m^{lk} (zeta_{2m}^{rk} U_k)              (Eq. (2.1))
//   2m U_k   = sum_r zeta_{2m}^{-rk} sum_l zeta_m^{-lk} u_{2l+r}   (Eq. (2.2))
// so per residue: twiddle the inputs, two backward m-point transforms, the
// pointwise product, one forward m-point transform, and the twiddled
// accumulation into the output.
//
// Level 1 (m <= 256 E): one thread group of T = m/E threads per instance,
// both arrays in shared memory.  Stockham stages with natural order in and
// out; the forward transform uses the backward radices in reverse order, so
// the last backward stage and the first forward stage touch the same
// thread-private positions and the product happens in registers between
// them.
//
// Level 2 (m = L1 * L2): the m-point transform as L1-point row transforms
// and L2-point column transforms (the two-factor split of a DFT):
//   pass A (column tile): for both residues and both inputs, the L2-point
//       backward transforms of the columns k1, written row-major to
//       scratch S[j2][k1];
//   pass B (row group): rows j2 of one residue: times zeta_m^{j2 k1},
//       L1-point backward transforms of the f and g rows, product,
//       L1-point forward transform, times zeta_m^{-j2 k1}, written back
//       over the f row;
//   pass C (column tile): for both residues, the L2-point forward
//       transforms of the product columns, then the residue
//       recombination (Eq. (2.2)) into the output.
// The scratch of a pass stays in L2; the passes are separate tasks of the
// persistent queue (fixed_batched.cu).
#pragma once

#include "fft2.cuh"

// The engine is compiled once per precision: DC_FX_P names the namespace
// (f32 / f64) and DC_FX_C the complex type (float2 / double2).
#ifndef DC_FX_P
#define DC_FX_P f32
#define DC_FX_C float2
#endif

namespace dc {
namespace fx {
namespace DC_FX_P {

constexpr int kThreads = 256;    // threads per block (FP32: two blocks per SM, FP64: one)
constexpr int kRootsMax = 768;   // shared-memory root entries reserved (2m <= 131072)

using C = DC_FX_C;
using Real = decltype(C{}.x);
constexpr bool kDouble = sizeof(C) == 16;

// ---------------------------------------------------------------------------
// compile-time plans
// ---------------------------------------------------------------------------
struct Plan {
  int n;
  int r[12];
};

__host__ __device__ constexpr int odd_part(int L) { return L % 5 == 0 ? 5 : (L % 3 == 0 ? 3 : 1); }
__host__ __device__ constexpr int pow2_cap(int E) {
  int c = 1;
  while (c < 16 && E % (2 * c) == 0) c *= 2;
  return c;
}
// radices of an L-point transform with E elements per thread: the largest
// power of two dividing E (at most 16) repeatedly, the remaining power of
// two, then the odd factor, merged with the power of two that completes E
// into one compound radix (24 = 8 x 3, 20 = 4 x 5) when L allows it
__host__ __device__ constexpr Plan make_plan(int L, int E) {
  Plan p{0, {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0}};
  const int odd = odd_part(L);
  int rest = L / odd;
  int last = odd;
  if (odd > 1 && E % odd == 0 && rest % (E / odd) == 0) {
    last = E;
    rest /= E / odd;
  }
  const int cap = pow2_cap(E);
  while (rest > 1) {
    const int r = rest >= cap ? cap : rest;
    p.r[p.n++] = r;
    rest /= r;
  }
  if (last > 1) p.r[p.n++] = last;
  return p;
}
// elements per thread of the row/level-1 transforms of a size family
__host__ __device__ constexpr int family_E(int L) {
  return odd_part(L) == 1 ? 16 : (odd_part(L) == 3 ? 24 : 20);
}
__host__ __device__ constexpr bool is_level1(int m) { return m <= kThreads * family_E(m); }
// Two-level split m = L1 L2 (L2: the column transforms' length).  Variant 0
// takes L2 = 128 up to m = 32768 and 256 above; variant 1 takes 64 for the
// smallest two-level size of each family (8192, 12288, 10240) and
// otherwise the other one of 128 and 256 (the autotuner picks per size,
// FP32 binary complex plans only).
__host__ __device__ constexpr int l2_cols(int m, int v = 0) {
  return v == 0 ? (m <= 32768 ? 128 : 256) : (m <= 12288 ? 64 : (m <= 32768 ? 256 : 128));
}
__host__ __device__ constexpr int l2_rows(int m, int v = 0) { return m / l2_cols(m, v); }   // L1
// column transforms: 16 elements per thread where the tile width divides
// the row length, else 8; tile width W = columns per block-wide tile
__host__ __device__ constexpr int col_E(int m, int v = 0) {
  return l2_rows(m, v) % (kThreads * 16 / l2_cols(m, v)) == 0 ? 16 : 8;
}
__host__ __device__ constexpr int col_width(int m, int v = 0) { return kThreads * col_E(m, v) / l2_cols(m, v); }
__host__ __device__ constexpr int padded(int L) { return (L + (L >> 4) + 2) & ~1; }
// Element stride between the array pairs (A, B) of consecutive thread groups
// of T threads.  When several groups share a half-warp (T < 16) the stride
// is made congruent to T modulo 16, so the groups' contiguous runs fall on
// disjoint bank pairs instead of the same ones.
__host__ __device__ constexpr int group_stride(int L, int T) {
  return T >= 16 ? 2 * padded(L) : 2 * padded(L) + ((T - 2 * padded(L)) % 16 + 16) % 16;
}

template <int L, int E> struct Fft {
  static constexpr Plan P = make_plan(L, E);
  static constexpr int n = P.n;
  static constexpr int T = L / E;
  // backward stages use the radices in plan order, forward stages in reverse
  __host__ __device__ static constexpr int radix(bool fwd, int s) { return fwd ? P.r[n - 1 - s] : P.r[s]; }
  __host__ __device__ static constexpr int ns(bool fwd, int s) {
    int x = 1;
    for (int t = 0; t < s; ++t) x *= radix(fwd, t);
    return x;
  }
};

template <int L, int E, int S, bool FWD> struct Stage {
  using F = Fft<L, E>;
  static constexpr int R = F::radix(FWD, S);
  static constexpr int Ns = F::ns(FWD, S);
  static constexpr int NB = E / R;
  static constexpr int LR = L / R;
  static constexpr int T = F::T;
  static_assert(E % R == 0, "radix must divide E");
};

// ---------------------------------------------------------------------------
// stage-twiddle tables.  Stage s of a transform multiplies input q of the
// butterfly at j by zeta_{Ns R}^{q k}, k = j mod Ns.  For every twiddled
// stage with Ns R <= kTabP the engine keeps these factors in shared memory
// as a table of R - 1 rows of Ns entries (row q - 1, column k), filled from
// the root table when a block switches to a size: one load per factor
// instead of forming the powers of zeta_{Ns R}^k by products, and the
// threads of a warp read consecutive (or equal) entries of a row, so the
// loads meet no bank conflicts.  The tables of a transform (L, E) list its
// distinct (Ns, R) over both directions (the forward transform runs the
// radices in reverse order).
// ---------------------------------------------------------------------------
constexpr int kTabP = 512;
struct TabLayout {
  int n;
  int ns[24], r[24], off[24];
  int total;   // entries
};
// Shared memory a block may use: two blocks per SM in FP32, one in FP64
// (228 KB per SM less 1 KB reserved per block and the static variables).
constexpr int kBlockSmemMax = kDouble ? 233472 - 1024 - 64 : (233472 - 2 * 1024) / 2 - 64;
template <int L, int E> struct StageTab {
  // A one-level transform (L, E) of the batched kernel takes its whole block:
  // kThreads / (L / E) instances in padded shared arrays behind the root
  // reservation.  Its tables go behind those, and are left out (the
  // twiddles formed by products instead) where they would not fit.
  static constexpr bool fits(int total) {
    return !(E == family_E(L) && is_level1(L)) ||
           kRootsMax * (int)sizeof(C) + (kThreads / (L / E)) * group_stride(L, L / E) * (int)sizeof(C) + 16 +
                   total * (int)sizeof(C) <=
               kBlockSmemMax;
  }
  static constexpr TabLayout make() {
    TabLayout t{};
    using F = Fft<L, E>;
    for (int d = 0; d < 2; ++d)
      for (int s = 1; s < F::n; ++s) {
        const int ns = F::ns(d == 1, s), r = F::radix(d == 1, s);
        if (ns * r > kTabP) continue;
        bool seen = false;
        for (int x = 0; x < t.n; ++x) seen = seen || (t.ns[x] == ns && t.r[x] == r);
        if (seen) continue;
        t.ns[t.n] = ns;
        t.r[t.n] = r;
        t.off[t.n] = t.total;
        t.total += (r - 1) * ns;
        ++t.n;
      }
    if (!fits(t.total)) t = TabLayout{};
    return t;
  }
  static constexpr TabLayout lay = make();
  // entry offset of the table of (Ns, R), -1 when the stage has none
  static constexpr int find(int ns, int r) {
    for (int x = 0; x < lay.n; ++x)
      if (lay.ns[x] == ns && lay.r[x] == r) return lay.off[x];
    return -1;
  }
};

// The root tables plus the stage tables of one transform (st: its first
// entry).  Code given a plain Roots<C> forms every stage twiddle from the
// root table instead.
struct TabRoots : Roots<C> {
  const C* st;
};
template <class RT, int L, int E, int NS, int R> struct TabOf {
  static constexpr int off = -1;
};
template <int L, int E, int NS, int R> struct TabOf<TabRoots, L, E, NS, R> {
  static constexpr int off = StageTab<L, E>::find(NS, R);
};

// Writes the stage tables of transform (L, E) at st (device memory; one
// block of kThreads threads): zeta_{Ns R}^{q k} computed in FP64 with
// sincospi from the exponent q k mod Ns R, then rounded.
template <int L, int E>
__device__ __forceinline__ void gen_stage_tabs(C* st) {
  constexpr TabLayout t = StageTab<L, E>::lay;
#pragma unroll
  for (int x = 0; x < t.n; ++x) {
    const int ns = t.ns[x], p = ns * t.r[x];
    for (int e = threadIdx.x; e < (t.r[x] - 1) * ns; e += kThreads) {
      const int q = 1 + e / ns, k = e - (q - 1) * ns;
      double sn, cs;
      sincospi(2.0 * (double)((q * k) % p) / (double)p, &sn, &cs);
      st[t.off[x] + e].x = (Real)cs;
      st[t.off[x] + e].y = (Real)sn;
    }
  }
}

// ---------------------------------------------------------------------------
// compound radices R = A B (12 = 4 x 3, 20 = 4 x 5, 24 = 8 x 3) as nested
// DFTs in registers: with n = B n1 + n2 and k = k1 + A k2,
//   X[k1 + A k2] = sum_{n2} zeta_B^{n2 k2} zeta_R^{n2 k1} sum_{n1} zeta_A^{n1 k1} x[B n1 + n2]
// (the Cooley-Tukey split of a DFT; internal twiddles are constants).
// ---------------------------------------------------------------------------
template <int R> struct RootConst;
template <> struct RootConst<12> {
  static constexpr double c[12] = {1.0, 0.86602540378443871, 0.5, 0.0, -0.5, -0.86602540378443871, -1.0, -0.86602540378443882, -0.5, 0.0, 0.5, 0.86602540378443837};
  static constexpr double s[12] = {0.0, 0.5, 0.8660254037844386, 1.0, 0.86602540378443871, 0.5, 0.0, -0.5, -0.86602540378443837, -1.0, -0.8660254037844386, -0.5};
};
template <> struct RootConst<20> {
  static constexpr double c[20] = {1.0, 0.95105651629515353, 0.80901699437494745, 0.58778525229247314, 0.30901699437494745, 0.0, -0.30901699437494734, -0.58778525229247303, -0.80901699437494734, -0.95105651629515353, -1.0, -0.95105651629515375, -0.80901699437494756, -0.58778525229247325, -0.30901699437494756, 0.0, 0.30901699437494723, 0.58778525229247292, 0.80901699437494734, 0.95105651629515353};
  static constexpr double s[20] = {0.0, 0.3090169943749474, 0.58778525229247314, 0.80901699437494745, 0.95105651629515353, 1.0, 0.95105651629515364, 0.80901699437494745, 0.58778525229247325, 0.30901699437494751, 0.0, -0.3090169943749469, -0.58778525229247303, -0.80901699437494734, -0.95105651629515353, -1.0, -0.95105651629515364, -0.80901699437494756, -0.58778525229247336, -0.30901699437494762};
};
template <> struct RootConst<24> {
  static constexpr double c[24] = {1.0, 0.96592582628906831, 0.86602540378443871, 0.70710678118654757, 0.5, 0.25881904510252074, 0.0, -0.25881904510252063, -0.5, -0.70710678118654746, -0.86602540378443871, -0.9659258262890682, -1.0, -0.96592582628906831, -0.86602540378443882, -0.70710678118654791, -0.5, -0.25881904510252063, 0.0, 0.2588190451025203, 0.5, 0.70710678118654735, 0.86602540378443837, 0.96592582628906809};
  static constexpr double s[24] = {0.0, 0.25881904510252074, 0.5, 0.70710678118654746, 0.8660254037844386, 0.96592582628906831, 1.0, 0.96592582628906831, 0.86602540378443871, 0.70710678118654757, 0.5, 0.25881904510252102, 0.0, -0.25881904510252079, -0.5, -0.70710678118654713, -0.86602540378443837, -0.96592582628906831, -1.0, -0.96592582628906842, -0.8660254037844386, -0.70710678118654768, -0.5, -0.25881904510252157};
};

// x * zeta_R^{sgn K}, exact for multiples of a quarter turn
template <int R, int K>
__device__ __forceinline__ C mul_root(C x, int sgn) {
  constexpr int k = ((K % R) + R) % R;
  if constexpr (k == 0) {
    return x;
  } else if constexpr (4 * k == R) {
    return si(x, sgn);
  } else if constexpr (2 * k == R) {
    C y;
    y.x = -x.x;
    y.y = -x.y;
    return y;
  } else if constexpr (4 * k == 3 * R) {
    return si(x, -sgn);
  } else {
    constexpr Real c = (Real)RootConst<R>::c[k], s = (Real)RootConst<R>::s[k];
    return mcs(x, c, s, sgn);
  }
}

template <int A, int B, int R, int K1, int N2>
__device__ __forceinline__ void nested_tw(C (&y)[A][B], int sgn) {
  if constexpr (K1 < A) {
    if constexpr (N2 < B) {
      y[K1][N2] = mul_root<R, K1 * N2>(y[K1][N2], sgn);
      nested_tw<A, B, R, K1, N2 + 1>(y, sgn);
    } else {
      nested_tw<A, B, R, K1 + 1, 0>(y, sgn);
    }
  }
}

template <int A, int B>
__device__ __forceinline__ void rdft_nested(C* x, int sgn) {
  constexpr int R = A * B;
  C y[A][B];
  C t[A];
#pragma unroll
  for (int n2 = 0; n2 < B; ++n2) {
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) t[n1] = x[B * n1 + n2];
    rdft<A>(t, sgn);
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) y[k1][n2] = t[k1];
  }
  nested_tw<A, B, R, 0, 0>(y, sgn);
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1) {
    C u[B];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) u[n2] = y[k1][n2];
    rdft<B>(u, sgn);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) x[k1 + A * k2] = u[k2];
  }
}

// radix-R DFT of the fixed engine: the shared butterflies, or a nested one
template <int R>
__device__ __forceinline__ void rdft_fx(C* x, int sgn) {
  if constexpr (R == 12) rdft_nested<4, 3>(x, sgn);
  else if constexpr (R == 20) rdft_nested<4, 5>(x, sgn);
  else if constexpr (R == 24) rdft_nested<8, 3>(x, sgn);
  else rdft<R>(x, sgn);
}

// ---------------------------------------------------------------------------
// shared-memory layouts
// ---------------------------------------------------------------------------
struct Contig {   // element x at p[x + x/16]: 16 elements span the 32 banks, one pad word pair
  C* p;
  __device__ __forceinline__ C& operator[](int x) const { return p[x + (x >> 4)]; }
};
template <int W> struct Inter {   // column tile: element x of this column at p[x * W]
  C* p;
  __device__ __forceinline__ C& operator[](int x) const { return p[x * W]; }
};

// ---------------------------------------------------------------------------
// barriers between stages: the threads that share the arrays, no more.
// A group of at most 32 threads lies within one warp (__syncwarp); a larger
// group that is not the whole block uses its own named barrier (id 1 + its
// index; 0 is the block barrier).
// ---------------------------------------------------------------------------
struct BlockSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
template <int T> struct GroupSync {
  int id;
  __device__ __forceinline__ void operator()() const {
    if constexpr (T >= kThreads) {
      __syncthreads();
    } else if constexpr (T <= 32) {
      __syncwarp();
    } else {
      static_assert(T % 32 == 0 && kThreads / T < 16, "named barriers cover whole warps");
      asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(T) : "memory");
    }
  }
};

// ---------------------------------------------------------------------------
// stage pieces
// ---------------------------------------------------------------------------
// v[b R + q] = X[i + b T + q L/R]
template <int L, int E, int S, bool FWD, class Lay>
__device__ __forceinline__ void gather(C* v, int i, const Lay& X) {
  using K = Stage<L, E, S, FWD>;
#pragma unroll
  for (int b = 0; b < K::NB; ++b)
#pragma unroll
    for (int q = 0; q < K::R; ++q) v[b * K::R + q] = X[i + b * K::T + q * K::LR];
}

// X[(j - k) R + k + q Ns] = v[b R + q], j = i + b T, k = j mod Ns
template <int L, int E, int S, bool FWD, class Lay>
__device__ __forceinline__ void scatter(const C* v, int i, const Lay& X) {
  using K = Stage<L, E, S, FWD>;
#pragma unroll
  for (int b = 0; b < K::NB; ++b) {
    const int j = i + b * K::T;
    const int k = j % K::Ns;
#pragma unroll
    for (int q = 0; q < K::R; ++q) X[(j - k) * K::R + k + q * K::Ns] = v[b * K::R + q];
  }
}

// Multiplies x[q] (q = 1 .. R-1) by w^q (FWD: conj(w)^q), w = zeta_TN^e,
// with the powers formed from exact table values at q = 1, 4, 8, 16 (those
// below R) by products of depth at most four: w2 = w1^2, w3 = w2 w1,
// w12 = w8 w4, w20 = w16 w4, w_{4a+b} = w_{4a} w_b.  A few table lookups per
// butterfly instead of R - 1, and each power is applied as soon as it is
// formed, so only w1, w2, w3 and the current w_{4a} stay live.
template <int R, bool FWD>
__device__ __forceinline__ void tw_apply(C* x, const Roots<C>& rt, int e) {
  auto app = [&](int q, C w) { x[q] = FWD ? cmulc(x[q], w) : cmul(x[q], w); };
  const C w1 = rt.at(e);
  app(1, w1);
  C w2 = w1, w3 = w1;
  if constexpr (R > 2) { w2 = cmul(w1, w1); app(2, w2); }
  if constexpr (R > 3) { w3 = cmul(w2, w1); app(3, w3); }
  if constexpr (R == 5) app(4, cmul(w2, w2));
  if constexpr (R > 5) {
    C w4 = w1, w8 = w1, w16 = w1;
#pragma unroll
    for (int a = 1; 4 * a < R; ++a) {
      C wa;
      if (a == 1) wa = w4 = rt.at(4 * e);
      else if (a == 2) wa = w8 = rt.at(8 * e);
      else if (a == 4) wa = w16 = rt.at(16 * e);
      else if (a == 3) wa = cmul(w8, w4);
      else wa = cmul(w16, w4);   // a == 5
      app(4 * a, wa);
      if (4 * a + 1 < R) app(4 * a + 1, cmul(wa, w1));
      if (4 * a + 2 < R) app(4 * a + 2, cmul(wa, w2));
      if (4 * a + 3 < R) app(4 * a + 3, cmul(wa, w3));
    }
  }
}

// twiddles zeta_{Ns R}^{+-q k} (root table of zeta_TN) and the radix-R DFT
// of each butterfly; backward: +, forward: -
template <int L, int E, int S, bool FWD, int TN, class RT>
__device__ __forceinline__ void dft(C* v, int i, const RT& rt) {
  using K = Stage<L, E, S, FWD>;
  constexpr int sgn = FWD ? -1 : 1;
  constexpr int toff = K::Ns > 1 ? TabOf<RT, L, E, K::Ns, K::R>::off : -1;
#pragma unroll
  for (int b = 0; b < K::NB; ++b) {
    if constexpr (K::Ns > 1) {
      static_assert(TN % (K::Ns * K::R) == 0, "root table must cover the stage");
      const int j = i + b * K::T;
      if constexpr (toff >= 0) {
        // row q - 1 of the stage table, column k = j mod Ns
        const C* t = rt.st + toff + j % K::Ns;
        C* x = &v[b * K::R];
#pragma unroll
        for (int q = 1; q < K::R; ++q) {
          const C w = t[(q - 1) * K::Ns];
          x[q] = FWD ? cmulc(x[q], w) : cmul(x[q], w);
        }
      } else {
        tw_apply<K::R, FWD>(&v[b * K::R], rt, (j % K::Ns) * (TN / (K::Ns * K::R)));
      }
    }
    rdft_fx<K::R>(&v[b * K::R], sgn);
  }
}

// natural index of element (b, q) of stage S's gather pattern
template <int L, int E, int S, bool FWD>
__device__ __forceinline__ int pos(int i, int b, int q) {
  using K = Stage<L, E, S, FWD>;
  return i + b * K::T + q * K::LR;
}

// ---------------------------------------------------------------------------
// one residue of a convolution of length L on a thread group (level 1 and
// the rows of pass B).  ld(x, arr, e) gives input arr (0: f, 1: g) at natural
// index x (register e), already twiddled for the residue; arr 0 comes first; st(x, v) takes the forward
// transform's output at natural index x (e: its register index).  A and B: padded shared arrays of
// the group.  Every thread of the block calls this (barriers inside).
// ---------------------------------------------------------------------------
template <int L, int E, int TN, int S, class RT, class Sy>
__device__ __forceinline__ void bwd_middle(C* v, int i, bool act, const Contig& A, const Contig& B,
                                           const RT& rt, const Sy& sync) {
  constexpr int n = Fft<L, E>::n;
  if constexpr (S < n - 1) {
    if (act) {
      gather<L, E, S, false>(v, i, A);
      dft<L, E, S, false, TN>(v, i, rt);
    }
    sync();
    if (act) {
      scatter<L, E, S, false>(v, i, A);
      gather<L, E, S, false>(v, i, B);
      dft<L, E, S, false, TN>(v, i, rt);
    }
    sync();
    if (act) scatter<L, E, S, false>(v, i, B);
    bwd_middle<L, E, TN, S + 1>(v, i, act, A, B, rt, sync);
  }
}

// middle stages of one array in place (gather, barrier, scatter, barrier)
template <int L, int E, int TN, bool FWD, int S, class Lay, class RT, class Sy>
__device__ __forceinline__ void one_middle(C* v, int i, bool act, const Lay& A, const RT& rt,
                                           const Sy& sync) {
  constexpr int n = Fft<L, E>::n;
  if constexpr (S < n - 1) {
    if (act) {
      gather<L, E, S, FWD>(v, i, A);
      dft<L, E, S, FWD, TN>(v, i, rt);
    }
    sync();
    if (act) scatter<L, E, S, FWD>(v, i, A);
    sync();
    one_middle<L, E, TN, FWD, S + 1>(v, i, act, A, rt, sync);
  }
}

// pointwise product of the two transformed arrays (binary complex case)
struct CProd {
  __device__ __forceinline__ C operator()(C a, C b) const { return cmul(a, b); }
};

template <int L, int E, int TN, class RT, class Ld, class St, class Sy, class Pr = CProd>
__device__ __forceinline__ void conv_residue(int i, bool act, C* Ap, C* Bp, const RT& rt,
                                             const Ld& ld, const St& st, const Sy& sync,
                                             const Pr& prod = Pr{}) {
  using F = Fft<L, E>;
  constexpr int n = F::n;
  static_assert(n >= 2, "at least two stages");
  const Contig A{Ap}, B{Bp};
  C v[E];
  // backward stage 0 of both inputs, straight from the source
  if (act) {
#pragma unroll
    for (int arr = 0; arr < 2; ++arr) {
      using K = Stage<L, E, 0, false>;
#pragma unroll
      for (int b = 0; b < K::NB; ++b)
#pragma unroll
        for (int q = 0; q < K::R; ++q) v[b * K::R + q] = ld(pos<L, E, 0, false>(i, b, q), arr, b * K::R + q);
      dft<L, E, 0, false, TN>(v, i, rt);
      scatter<L, E, 0, false>(v, i, arr ? B : A);
    }
  }
  sync();
  bwd_middle<L, E, TN, 1>(v, i, act, A, B, rt, sync);
  // last backward stage: thread-private positions (k = j), in place
  if (act) {
    gather<L, E, n - 1, false>(v, i, A);
    dft<L, E, n - 1, false, TN>(v, i, rt);
    scatter<L, E, n - 1, false>(v, i, A);
  }
  if constexpr (n > 2) sync();
  if (act) {
    gather<L, E, n - 1, false>(v, i, B);
    dft<L, E, n - 1, false, TN>(v, i, rt);
    // pointwise product with the f values at the same positions
    using K = Stage<L, E, n - 1, false>;
#pragma unroll
    for (int b = 0; b < K::NB; ++b)
#pragma unroll
      for (int q = 0; q < K::R; ++q)
        v[b * K::R + q] = prod(A[pos<L, E, n - 1, false>(i, b, q)], v[b * K::R + q]);
    // first forward stage: same radix and positions, no twiddles
    dft<L, E, 0, true, TN>(v, i, rt);
  }
  sync();
  if (act) scatter<L, E, 0, true>(v, i, A);
  sync();
  one_middle<L, E, TN, true, 1>(v, i, act, A, rt, sync);
  // last forward stage: thread-private positions
  if (act) {
    gather<L, E, n - 1, true>(v, i, A);
    dft<L, E, n - 1, true, TN>(v, i, rt);
    using K = Stage<L, E, n - 1, true>;
#pragma unroll
    for (int b = 0; b < K::NB; ++b)
#pragma unroll
      for (int q = 0; q < K::R; ++q) st(pos<L, E, n - 1, true>(i, b, q), b * K::R + q, v[b * K::R + q]);
  }
}

// ---------------------------------------------------------------------------
// one residue of a centered Hermitian convolution (Sec. 2.3) on a thread
// group: a single array holds w^f + i w^g (both transforms are real), so
// one backward transform gives u^f (real part) and u^g (imaginary part);
// their product, a real array, takes one forward transform.  ld(x, e) gives
// the packed input at natural index x; st(x, e, v) takes the output.
// ---------------------------------------------------------------------------
template <int L, int E, int TN, class RT, class Ld, class St, class Sy>
__device__ __forceinline__ void conv1_residue(int i, C* Ap, const RT& rt, const Ld& ld, const St& st,
                                              const Sy& sync) {
  using F = Fft<L, E>;
  constexpr int n = F::n;
  static_assert(n >= 2, "at least two stages");
  const Contig A{Ap};
  C v[E];
  {
    using K = Stage<L, E, 0, false>;
#pragma unroll
    for (int b = 0; b < K::NB; ++b)
#pragma unroll
      for (int q = 0; q < K::R; ++q) v[b * K::R + q] = ld(pos<L, E, 0, false>(i, b, q), b * K::R + q);
  }
  dft<L, E, 0, false, TN>(v, i, rt);
  scatter<L, E, 0, false>(v, i, A);
  sync();
  one_middle<L, E, TN, false, 1>(v, i, true, A, rt, sync);
  // last backward stage (thread-private positions), the real product and
  // the first forward stage in registers
  gather<L, E, n - 1, false>(v, i, A);
  dft<L, E, n - 1, false, TN>(v, i, rt);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    v[e].x = v[e].x * v[e].y;
    v[e].y = 0;
  }
  dft<L, E, 0, true, TN>(v, i, rt);
  sync();
  scatter<L, E, 0, true>(v, i, A);
  sync();
  one_middle<L, E, TN, true, 1>(v, i, true, A, rt, sync);
  gather<L, E, n - 1, true>(v, i, A);
  dft<L, E, n - 1, true, TN>(v, i, rt);
  using KF = Stage<L, E, n - 1, true>;
#pragma unroll
  for (int b = 0; b < KF::NB; ++b)
#pragma unroll
    for (int q = 0; q < KF::R; ++q) st(pos<L, E, n - 1, true>(i, b, q), b * KF::R + q, v[b * KF::R + q]);
}

// ---------------------------------------------------------------------------
// one residue of the rows of a centered Hermitian gradient (two Hermitian
// convolutions sharing W, Sec. 2.3 applied to the adjoint): array A takes
// W's packed input (its transform is real; the real part is kept), array B
// w^f + i w^g.  The real products a = u^W u^g (output 0) and b = u^W u^f
// (output 1) share one forward transform Y of a + i b; since both are
// real, their transforms are (Y_k + conj Y_{L-k}) / 2 and
// (Y_k - conj Y_{L-k}) / 2i, read back through A.  ld(x, arr, e) gives
// input arr at natural index x; st(x, e, v, o) takes output o.
// ---------------------------------------------------------------------------
template <int L, int E, int TN, class RT, class Ld, class St, class Sy>
__device__ __forceinline__ void conv_pair_residue(int i, C* Ap, C* Bp, const RT& rt, const Ld& ld,
                                                  const St& st, const Sy& sync) {
  using F = Fft<L, E>;
  constexpr int n = F::n;
  static_assert(n >= 2, "at least two stages");
  const Contig A{Ap}, B{Bp};
  C v[E];
#pragma unroll
  for (int arr = 0; arr < 2; ++arr) {
    using K = Stage<L, E, 0, false>;
#pragma unroll
    for (int b = 0; b < K::NB; ++b)
#pragma unroll
      for (int q = 0; q < K::R; ++q) v[b * K::R + q] = ld(pos<L, E, 0, false>(i, b, q), arr, b * K::R + q);
    dft<L, E, 0, false, TN>(v, i, rt);
    scatter<L, E, 0, false>(v, i, arr ? B : A);
  }
  sync();
  bwd_middle<L, E, TN, 1>(v, i, true, A, B, rt, sync);
  gather<L, E, n - 1, false>(v, i, A);
  dft<L, E, n - 1, false, TN>(v, i, rt);
  scatter<L, E, n - 1, false>(v, i, A);
  if constexpr (n > 2) sync();
  gather<L, E, n - 1, false>(v, i, B);
  dft<L, E, n - 1, false, TN>(v, i, rt);
  using KB = Stage<L, E, n - 1, false>;
#pragma unroll
  for (int b = 0; b < KB::NB; ++b)
#pragma unroll
    for (int q = 0; q < KB::R; ++q) {
      const int x = pos<L, E, n - 1, false>(i, b, q), e = b * KB::R + q;
      const Real uw = A[x].x;
      const Real uf = v[e].x;
      v[e].x = uw * v[e].y;   // u^W u^g
      v[e].y = uw * uf;       // u^W u^f
    }
  dft<L, E, 0, true, TN>(v, i, rt);
  sync();
  scatter<L, E, 0, true>(v, i, A);
  sync();
  one_middle<L, E, TN, true, 1>(v, i, true, A, rt, sync);
  gather<L, E, n - 1, true>(v, i, A);
  dft<L, E, n - 1, true, TN>(v, i, rt);
  using KF = Stage<L, E, n - 1, true>;
  sync();
#pragma unroll
  for (int b = 0; b < KF::NB; ++b)
#pragma unroll
    for (int q = 0; q < KF::R; ++q) A[pos<L, E, n - 1, true>(i, b, q)] = v[b * KF::R + q];
  sync();
#pragma unroll
  for (int b = 0; b < KF::NB; ++b)
#pragma unroll
    for (int q = 0; q < KF::R; ++q) {
      const int x = pos<L, E, n - 1, true>(i, b, q), e = b * KF::R + q;
      const C y = v[e], ym = A[x ? L - x : 0];
      C o0, o1;
      o0.x = (Real)0.5 * (y.x + ym.x);
      o0.y = (Real)0.5 * (y.y - ym.y);
      o1.x = (Real)0.5 * (y.y + ym.y);
      o1.y = (Real)0.5 * (ym.x - y.x);
      st(x, e, o0, 0);
      st(x, e, o1, 1);
    }
}

// ---------------------------------------------------------------------------
// one L-point column transform of a tile (passes A and C).  v holds the
// inputs of stage 0 in gather order; st(x, e, v) takes output x (register e).  D: this
// thread's column of the interleaved tile.  Every thread calls this.
// ---------------------------------------------------------------------------
template <int L, int E, int W, int TN, bool FWD, class RT, class St>
__device__ __forceinline__ void column(C* v, int i, C* Dp, const RT& rt, const St& st) {
  constexpr int n = Fft<L, E>::n;
  static_assert(n >= 2, "at least two stages");
  const Inter<W> D{Dp};
  dft<L, E, 0, FWD, TN>(v, i, rt);
  scatter<L, E, 0, FWD>(v, i, D);
  __syncthreads();
  one_middle<L, E, TN, FWD, 1>(v, i, true, D, rt, BlockSync{});
  gather<L, E, n - 1, FWD>(v, i, D);
  dft<L, E, n - 1, FWD, TN>(v, i, rt);
  using K = Stage<L, E, n - 1, FWD>;
#pragma unroll
  for (int b = 0; b < K::NB; ++b)
#pragma unroll
    for (int q = 0; q < K::R; ++q) st(pos<L, E, n - 1, FWD>(i, b, q), b * K::R + q, v[b * K::R + q]);
}

}  // namespace DC_FX_P
}  // namespace fx
}  // namespace dc

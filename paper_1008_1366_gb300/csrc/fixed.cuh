// Fixed-shape engine: FP32 complex implicitly dealiased convolutions whose
// sizes are known at compile time.
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
//       backward transforms of the columns k1, times zeta_m^{j2 k1},
//       written row-major to scratch S[j2][k1];
//   pass B (row group): rows j2 of one residue: L1-point backward
//       transforms of the f and g rows, product, L1-point forward
//       transform, times zeta_m^{-j2 k1}, written back over the f row;
//   pass C (column tile): for both residues, the L2-point forward
//       transforms of the product columns, then the residue
//       recombination (Eq. (2.2)) into the output.
// The scratch of a pass stays in L2; the passes are separate tasks of the
// persistent queue (fixed_batched.cu).
#pragma once

#include "fft2.cuh"

namespace dc {
namespace fx {

constexpr int kThreads = 256;       // threads per block; two blocks per SM
constexpr int kRootsMax = 768;   // shared-memory root entries reserved (2m <= 131072)

using C = float2;

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
// two, then the odd factor
__host__ __device__ constexpr Plan make_plan(int L, int E) {
  Plan p{0, {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0}};
  const int odd = odd_part(L);
  int rest = L / odd;
  const int cap = pow2_cap(E);
  while (rest > 1) {
    const int r = rest >= cap ? cap : rest;
    p.r[p.n++] = r;
    rest /= r;
  }
  if (odd > 1) p.r[p.n++] = odd;
  return p;
}
// elements per thread of the row/level-1 transforms of a size family
__host__ __device__ constexpr int family_E(int L) {
  return odd_part(L) == 1 ? 16 : (odd_part(L) == 3 ? 24 : 20);
}
__host__ __device__ constexpr bool is_level1(int m) { return m <= kThreads * family_E(m); }
__host__ __device__ constexpr int l2_cols(int m) { return m <= 32768 ? 128 : 256; }   // L2
__host__ __device__ constexpr int l2_rows(int m) { return m / l2_cols(m); }           // L1
// column transforms: 16 elements per thread where the tile width divides
// the row length, else 8; tile width W = columns per block-wide tile
__host__ __device__ constexpr int col_E(int m) {
  return l2_rows(m) % (kThreads * 16 / l2_cols(m)) == 0 ? 16 : 8;
}
__host__ __device__ constexpr int col_width(int m) { return kThreads * col_E(m) / l2_cols(m); }
__host__ __device__ constexpr int padded(int L) { return (L + (L >> 4) + 2) & ~1; }

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

// Powers w[q] = w1^q, q < R, of a stage twiddle from exact table values of
// w1 and (R >= 8) w4 by products of depth at most three:
// w2 = w1^2, w3 = w2 w1, w8 = w4^2, w_{4a+b} = w_{4a} w_b.  Two table
// lookups per butterfly instead of R - 1.
template <int R>
__device__ __forceinline__ void tw_powers(C* w, C w1, C w4) {
  w[1] = w1;
  if constexpr (R > 2) w[2] = cmul(w1, w1);
  if constexpr (R > 3) w[3] = cmul(w[2], w1);
  if constexpr (R == 5) w[4] = cmul(w[2], w[2]);
  if constexpr (R >= 8) {
    w[4] = w4;
#pragma unroll
    for (int b = 1; b < 4; ++b) w[4 + b] = cmul(w4, w[b]);
  }
  if constexpr (R == 16) {
    const C w8 = cmul(w4, w4);
    const C w12 = cmul(w8, w4);
    w[8] = w8;
    w[12] = w12;
#pragma unroll
    for (int b = 1; b < 4; ++b) {
      w[8 + b] = cmul(w8, w[b]);
      w[12 + b] = cmul(w12, w[b]);
    }
  }
}

// twiddles zeta_{Ns R}^{+-q k} (root table of zeta_TN) and the radix-R DFT
// of each butterfly; backward: +, forward: -
template <int L, int E, int S, bool FWD, int TN>
__device__ __forceinline__ void dft(C* v, int i, const Roots<C>& rt) {
  using K = Stage<L, E, S, FWD>;
  constexpr int sgn = FWD ? -1 : 1;
#pragma unroll
  for (int b = 0; b < K::NB; ++b) {
    if constexpr (K::Ns > 1) {
      static_assert(TN % (K::Ns * K::R) == 0, "root table must cover the stage");
      const int j = i + b * K::T;
      const int e = (j % K::Ns) * (TN / (K::Ns * K::R));
      C w[K::R];
      tw_powers<K::R>(w, rt.at(e), K::R >= 8 ? rt.at(4 * e) : rt.at(0));
#pragma unroll
      for (int q = 1; q < K::R; ++q)
        v[b * K::R + q] = FWD ? cmulc(v[b * K::R + q], w[q]) : cmul(v[b * K::R + q], w[q]);
    }
    rdft<K::R>(&v[b * K::R], sgn);
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
template <int L, int E, int TN, int S>
__device__ __forceinline__ void bwd_middle(C* v, int i, bool act, const Contig& A, const Contig& B,
                                           const Roots<C>& rt) {
  constexpr int n = Fft<L, E>::n;
  if constexpr (S < n - 1) {
    if (act) {
      gather<L, E, S, false>(v, i, A);
      dft<L, E, S, false, TN>(v, i, rt);
    }
    __syncthreads();
    if (act) {
      scatter<L, E, S, false>(v, i, A);
      gather<L, E, S, false>(v, i, B);
      dft<L, E, S, false, TN>(v, i, rt);
    }
    __syncthreads();
    if (act) scatter<L, E, S, false>(v, i, B);
    bwd_middle<L, E, TN, S + 1>(v, i, act, A, B, rt);
  }
}

// middle stages of one array in place (gather, barrier, scatter, barrier)
template <int L, int E, int TN, bool FWD, int S, class Lay>
__device__ __forceinline__ void one_middle(C* v, int i, bool act, const Lay& A, const Roots<C>& rt) {
  constexpr int n = Fft<L, E>::n;
  if constexpr (S < n - 1) {
    if (act) {
      gather<L, E, S, FWD>(v, i, A);
      dft<L, E, S, FWD, TN>(v, i, rt);
    }
    __syncthreads();
    if (act) scatter<L, E, S, FWD>(v, i, A);
    __syncthreads();
    one_middle<L, E, TN, FWD, S + 1>(v, i, act, A, rt);
  }
}

template <int L, int E, int TN, class Ld, class St>
__device__ __forceinline__ void conv_residue(int i, bool act, C* Ap, C* Bp, const Roots<C>& rt,
                                             const Ld& ld, const St& st) {
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
  __syncthreads();
  bwd_middle<L, E, TN, 1>(v, i, act, A, B, rt);
  // last backward stage: thread-private positions (k = j), in place
  if (act) {
    gather<L, E, n - 1, false>(v, i, A);
    dft<L, E, n - 1, false, TN>(v, i, rt);
    scatter<L, E, n - 1, false>(v, i, A);
  }
  if constexpr (n > 2) __syncthreads();
  if (act) {
    gather<L, E, n - 1, false>(v, i, B);
    dft<L, E, n - 1, false, TN>(v, i, rt);
    // pointwise product with the f values at the same positions
    using K = Stage<L, E, n - 1, false>;
#pragma unroll
    for (int b = 0; b < K::NB; ++b)
#pragma unroll
      for (int q = 0; q < K::R; ++q)
        v[b * K::R + q] = cmul(A[pos<L, E, n - 1, false>(i, b, q)], v[b * K::R + q]);
    // first forward stage: same radix and positions, no twiddles
    dft<L, E, 0, true, TN>(v, i, rt);
  }
  __syncthreads();
  if (act) scatter<L, E, 0, true>(v, i, A);
  __syncthreads();
  one_middle<L, E, TN, true, 1>(v, i, act, A, rt);
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
// one L-point column transform of a tile (passes A and C).  v holds the
// inputs of stage 0 in gather order; st(x, e, v) takes output x (register e).  D: this
// thread's column of the interleaved tile.  Every thread calls this.
// ---------------------------------------------------------------------------
template <int L, int E, int W, int TN, bool FWD, class St>
__device__ __forceinline__ void column(C* v, int i, C* Dp, const Roots<C>& rt, const St& st) {
  constexpr int n = Fft<L, E>::n;
  static_assert(n >= 2, "at least two stages");
  const Inter<W> D{Dp};
  dft<L, E, 0, FWD, TN>(v, i, rt);
  scatter<L, E, 0, FWD>(v, i, D);
  __syncthreads();
  one_middle<L, E, TN, FWD, 1>(v, i, true, D, rt);
  gather<L, E, n - 1, FWD>(v, i, D);
  dft<L, E, n - 1, FWD, TN>(v, i, rt);
  using K = Stage<L, E, n - 1, FWD>;
#pragma unroll
  for (int b = 0; b < K::NB; ++b)
#pragma unroll
    for (int q = 0; q < K::R; ++q) st(pos<L, E, n - 1, FWD>(i, b, q), b * K::R + q, v[b * K::R + q]);
}

}  // namespace fx
}  // namespace dc

// Fused implicitly dealiased 1D convolutions.
//
// For each residue r of the padded index (j = q l + r), one block:
//   1. builds the r-th sub-transform inputs from the unpadded data
//      (pre-twiddle by zeta_{qm}^{rk}, Eq. (2.1); centered/Hermitian w_{k,r},
//      Eqs. (2.4)-(2.5) and Sec. 2.3; ternary zeta_{4m}^{rk} U_k, Sec. 4.2),
//   2. runs the m-point backward sub-transforms (fft.cuh),
//   3. forms the pointwise product,
//   4. runs the m-point forward sub-transform, and
//   5. accumulates zeta_{qm}^{-rk} times it into the output (Eq. (2.2),
//      Eqs. (2.6)/(2.7), Sec. 4.2); after the last residue the sum is scaled by
//      1/N and written.
// The padded array of size qm never exists: per residue only m-point arrays
// live in shared memory (level 1) or, for m beyond shared memory, in a
// per-block scratch slot that the two-level decomposition m = L1 * L2 streams
// through in column tiles and row tiles (level 2).
#pragma once

#include "fft.cuh"
#include "plan.h"

namespace dc {

constexpr int kThreads = 512;

struct ConvArgs {
  const void* in[3];      // inputs (f, g, e) or (w, f, g) for gradients
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

template <class C> __device__ __forceinline__ C twd(const C* tw, int i) { return __ldg(&tw[i]); }

// ---------------------------------------------------------------------------
// kind policies
// ---------------------------------------------------------------------------
template <int KIND, class C> struct KP;

// complex binary convolution, N = 2m, residues r = 0, 1 (Eqs. (2.1)-(2.2))
template <class C> struct KP<K_COMPLEX, C> {
  static constexpr int Q = 2, NARR = 2, NFWD = 1;
  __device__ static C build(const C* const* in, int x, int k, int ri, int m, const C* tw) {
    C v = in[x][k];
    return ri ? cmul(v, twd(tw, k)) : v;
  }
  __device__ static void pointwise(C* v) { v[0] = cmul(v[0], v[1]); }
  __device__ static C contrib(int, C X, int k, int ri, int m, const C* tw) {
    return ri ? cmulc(X, twd(tw, k)) : X;
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
__device__ __forceinline__ C herm_w(const C* u, int k, int r, int m, const C* tw, C x0) {
  using R = typename RealOf<C>::type;
  if (k == 0) return x0;
  C a = u[k];
  C b = cconj(u[m - k]);
  if (r == 0) return cadd(a, b);
  C z3; z3.x = (R)-0.5; z3.y = (R)(-r) * (R)0.86602540378443864676;
  a = cadd(a, cmul(b, z3));
  C t = twd(tw, k);
  return r > 0 ? cmul(a, t) : cmulc(a, t);
}

template <class C> __device__ __forceinline__ C pack_i(C a, C b) {  // a + i b
  C c; c.x = a.x - b.y; c.y = a.y + b.x; return c;
}

template <class C> __device__ __forceinline__ C herm_out_twiddle(C X, int k, int r, const C* tw) {
  // zeta_{3m}^{-rk} X (Eq. (2.7))
  if (r == 0) return X;
  C t = twd(tw, k);
  return r > 0 ? cmulc(X, t) : cmul(X, t);
}

template <class C> __device__ __forceinline__ C real_part(C a) { a.y = 0; return a; }

// centered Hermitian binary convolution, N = 3m, r = -1, 0, 1.  The two real
// backward transforms of f and g share one complex transform of
// w^f + i w^g (both results are real); the real product is forward
// transformed as a complex array with zero imaginary part.
template <class C> struct KP<K_HERMITIAN, C> {
  static constexpr int Q = 3, NARR = 1, NFWD = 1;
  __device__ static C build(const C* const* in, int, int k, int ri, int m, const C* tw) {
    const int r = ri - 1;
    C wf = herm_w(in[0], k, r, m, tw, real_part(in[0][0]));
    C wg = herm_w(in[1], k, r, m, tw, real_part(in[1][0]));
    return pack_i(wf, wg);
  }
  __device__ static void pointwise(C* v) { v[0].x = v[0].x * v[0].y; v[0].y = 0; }
  __device__ static C contrib(int, C X, int k, int ri, int, const C* tw) {
    return herm_out_twiddle(X, k, ri - 1, tw);
  }
  __device__ static C finish(int, C a, int, int m) {
    using R = typename RealOf<C>::type;
    return cscale(a, (R)1 / (R)(3 * m));
  }
};

// V_k of the ternary transform (Sec. 4.2): zeta_{4m}^{rk} U_k for k < m (U_0
// real), 0 at k = m, conj(V_{2m-k}) for m < k < 2m.
template <class C> __device__ __forceinline__ C tern_v(const C* u, int k, int r, int m, const C* tw) {
  if (k == m) { C z; z.x = 0; z.y = 0; return z; }
  const bool up = k > m;
  const int kk = up ? 2 * m - k : k;
  C x = u[kk];
  if (kk == 0) x.y = 0;
  if (r) x = cmul(x, twd(tw, kk));
  return up ? cconj(x) : x;
}

// centered Hermitian ternary convolution, N = 4m, r = 0, 1, sub-transforms of
// length 2m: (V^f + i V^g) and V^e backward, the triple real product forward.
template <class C> struct KP<K_TERNARY, C> {
  static constexpr int Q = 2, NARR = 2, NFWD = 1;
  __device__ static C build(const C* const* in, int x, int k, int ri, int m, const C* tw) {
    if (x == 0) return pack_i(tern_v(in[0], k, ri, m, tw), tern_v(in[1], k, ri, m, tw));
    return tern_v(in[2], k, ri, m, tw);
  }
  __device__ static void pointwise(C* v) { v[0].x = v[0].x * v[0].y * v[1].x; v[0].y = 0; }
  __device__ static C contrib(int, C X, int k, int ri, int, const C* tw) {
    return ri ? cmulc(X, twd(tw, k)) : X;
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
  __device__ static C build(const C* const* in, int x, int k, int ri, int m, const C* tw) {
    return KP<K_COMPLEX, C>::build(in, x, k, ri, m, tw);
  }
  __device__ static void pointwise(C* v) {
    C a = cmulc(v[0], v[2]);
    C b = cmulc(v[0], v[1]);
    v[0] = a; v[1] = b;
  }
  __device__ static C contrib(int o, C X, int k, int ri, int m, const C* tw) {
    return KP<K_COMPLEX, C>::contrib(o, X, k, ri, m, tw);
  }
  __device__ static C finish(int o, C a, int k, int m) { return KP<K_COMPLEX, C>::finish(o, a, k, m); }
};

// gradient of the Hermitian convolution: inputs (w, f, g).  W = w with
// W_0 = 2 Re w_0; df = S conv(W, g), dg = S conv(W, f) with S = 1/2 at k = 0.
// Backward: (W + i f) packed and g; forward: the two real products.
template <class C> struct KP<K_HERMITIAN_ADJ, C> {
  static constexpr int Q = 3, NARR = 2, NFWD = 2;
  __device__ static C build(const C* const* in, int x, int k, int ri, int m, const C* tw) {
    const int r = ri - 1;
    if (x == 0) {
      C w0 = real_part(in[0][0]);
      w0.x *= 2;
      C ww = herm_w(in[0], k, r, m, tw, w0);
      C wf = herm_w(in[1], k, r, m, tw, real_part(in[1][0]));
      return pack_i(ww, wf);
    }
    return herm_w(in[2], k, r, m, tw, real_part(in[2][0]));
  }
  __device__ static void pointwise(C* v) {
    const auto uw = v[0].x, uf = v[0].y, ug = v[1].x;
    v[0].x = uw * ug; v[0].y = 0;
    v[1].x = uw * uf; v[1].y = 0;
  }
  __device__ static C contrib(int, C X, int k, int ri, int, const C* tw) {
    return herm_out_twiddle(X, k, ri - 1, tw);
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
  __device__ static C build(const C* const* in, int x, int k, int ri, int m, const C* tw) {
    const int r = ri - 1;
    if (x == 0) {
      C ww = herm_w(in[0], k, r, m, tw, real_part(in[0][0]));
      C wf = herm_w(in[1], k, r, m, tw, real_part(in[1][0]));
      return pack_i(ww, wf);
    }
    return herm_w(in[2], k, r, m, tw, real_part(in[2][0]));
  }
  __device__ static void pointwise(C* v) { KP<K_HERMITIAN_ADJ, C>::pointwise(v); }
  __device__ static C contrib(int o, C X, int k, int ri, int m, const C* tw) {
    return KP<K_HERMITIAN_ADJ, C>::contrib(o, X, k, ri, m, tw);
  }
  __device__ static C finish(int o, C a, int k, int m) { return KP<K_HERMITIAN, C>::finish(o, a, k, m); }
};

// ---------------------------------------------------------------------------
// level 1: `count` instances of one size, each wholly in shared memory
// ---------------------------------------------------------------------------
template <int KIND, class C>
__device__ void conv_level1(const ConvArgs& a, const CfgDev& cfg, int first, int count, C* sm) {
  using K = KP<KIND, C>;
  const int L = cfg.L, m = cfg.m, TN = cfg.TN;
  const int tpt = cfg.p.tpt;
  const int t = threadIdx.x / tpt, i = threadIdx.x - t * tpt;
  const bool active = t < count;
  const C* tw = (const C*)cfg.tw;
  const C* in[3] = {nullptr, nullptr, nullptr};
  C* out[2] = {nullptr, nullptr};
  if (active) {
    const int inst = a.order ? a.order[first + t] : first + t;
    const int64_t off = a.off ? a.off[inst] : (int64_t)inst * a.stride;
#pragma unroll
    for (int x = 0; x < 3; ++x) if (a.in[x]) in[x] = (const C*)a.in[x] + off;
#pragma unroll
    for (int o = 0; o < 2; ++o) if (a.out[o]) out[o] = (C*)a.out[o] + off;
  }
  const int per = K::NARR * L + K::NFWD * m;
  C* base = sm + (size_t)(active ? t : 0) * per;
  C* acc = base + K::NARR * L;

  for (int ri = 0; ri < K::Q; ++ri) {
    if (active) {
#pragma unroll
      for (int x = 0; x < K::NARR; ++x)
        for (int k = i; k < L; k += tpt) base[x * L + k] = K::build(in, x, k, ri, m, tw);
    }
    __syncthreads();
#pragma unroll
    for (int x = 0; x < K::NARR; ++x) fft_smem<1>(base + x * L, 1, cfg.p, i, active, tw, TN);
    if (active) {
      for (int k = i; k < L; k += tpt) {
        C v[K::NARR];
#pragma unroll
        for (int x = 0; x < K::NARR; ++x) v[x] = base[x * L + k];
        K::pointwise(v);
#pragma unroll
        for (int o = 0; o < K::NFWD; ++o) base[o * L + k] = v[o];
      }
    }
    __syncthreads();
#pragma unroll
    for (int o = 0; o < K::NFWD; ++o) fft_smem<-1>(base + o * L, 1, cfg.p, i, active, tw, TN);
    if (active) {
#pragma unroll
      for (int o = 0; o < K::NFWD; ++o)
        for (int k = i; k < m; k += tpt) {
          C c = K::contrib(o, base[o * L + k], k, ri, m, tw);
          acc[o * m + k] = ri ? cadd(acc[o * m + k], c) : c;
        }
    }
    __syncthreads();
  }
  if (active) {
#pragma unroll
    for (int o = 0; o < K::NFWD; ++o)
      for (int k = i; k < m; k += tpt) out[o][k] = K::finish(o, acc[o * m + k], k, m);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// level 2: one instance, sub-transform L = L1 * L2 through a scratch slot.
// Backward DFT of length L with k = k1 + L1 k2, j = j2 + L2 j1:
//   pass A (column tiles): X[k1][j2] = sum_{k2} zeta_{L2}^{j2 k2} U[k1 + L1 k2],
//            times zeta_L^{j2 k1}, stored row-major S[j2][k1];
//   pass B (row tiles):    u[j2 + L2 j1] = sum_{k1} zeta_{L1}^{j1 k1} S[j2][k1];
//            pointwise product; the forward transform runs the same steps in
//            reverse: length-L1 forward DFT over j1, times zeta_L^{-j2 k1};
//   pass C (column tiles): length-L2 forward DFT over j2, then the residue
//            recombination into the output tile.
// The scrambled order between the halves is never undone (Sec. 1 notes bit
// reversal is unnecessary for a convolution).
// ---------------------------------------------------------------------------
template <int KIND, class C>
__device__ void conv_level2(const ConvArgs& a, const CfgDev& cfg, int first, C* sm, C* scr) {
  using K = KP<KIND, C>;
  const int L1 = cfg.L1, L2 = cfg.L2, L = cfg.L, m = cfg.m, TN = cfg.TN;
  const int w = cfg.w, nr = cfg.nr;
  const int tq = TN / L;
  const int T = blockDim.x, tid = threadIdx.x;
  const C* tw = (const C*)cfg.tw;
  const int inst = a.order ? a.order[first] : first;
  const int64_t off = a.off ? a.off[inst] : (int64_t)inst * a.stride;
  const C* in[3] = {nullptr, nullptr, nullptr};
  C* out[2] = {nullptr, nullptr};
#pragma unroll
  for (int x = 0; x < 3; ++x) if (a.in[x]) in[x] = (const C*)a.in[x] + off;
#pragma unroll
  for (int o = 0; o < 2; ++o) if (a.out[o]) out[o] = (C*)a.out[o] + off;

  const int cc = tid % w, ci = tid / w;
  const bool cact = ci < cfg.pc.tpt;
  const int tile = w * L2;

  // pass A
  for (int k1a = 0; k1a < L1; k1a += w) {
    for (int ri = 0; ri < K::Q; ++ri) {
#pragma unroll
      for (int x = 0; x < K::NARR; ++x) {
        for (int e = tid; e < tile; e += T) {
          const int c = e % w, k2 = e / w;
          sm[e] = K::build(in, x, k1a + c + L1 * k2, ri, m, tw);
        }
        __syncthreads();
        fft_smem<1>(sm + cc, w, cfg.pc, ci, cact, tw, TN);
        C* S = scr + (size_t)(ri * K::NARR + x) * L;
        for (int e = tid; e < tile; e += T) {
          const int c = e % w, j2 = e / w, k1 = k1a + c;
          S[(size_t)j2 * L1 + k1] = cmul(sm[e], twd(tw, j2 * k1 * tq));
        }
        __syncthreads();
      }
    }
  }
  // pass B
  const int rr = tid / cfg.pr.tpt, rj = tid - rr * cfg.pr.tpt;
  const bool ract = rr < nr;
  const int rtile = nr * L1;
  for (int j2a = 0; j2a < L2; j2a += nr) {
    for (int ri = 0; ri < K::Q; ++ri) {
#pragma unroll
      for (int x = 0; x < K::NARR; ++x) {
        const C* S = scr + (size_t)(ri * K::NARR + x) * L + (size_t)j2a * L1;
        for (int e = tid; e < rtile; e += T) sm[x * rtile + e] = S[e];
      }
      __syncthreads();
#pragma unroll
      for (int x = 0; x < K::NARR; ++x)
        fft_smem<1>(sm + x * rtile + rr * L1, 1, cfg.pr, rj, ract, tw, TN);
      for (int e = tid; e < rtile; e += T) {
        C v[K::NARR];
#pragma unroll
        for (int x = 0; x < K::NARR; ++x) v[x] = sm[x * rtile + e];
        K::pointwise(v);
#pragma unroll
        for (int o = 0; o < K::NFWD; ++o) sm[o * rtile + e] = v[o];
      }
      __syncthreads();
#pragma unroll
      for (int o = 0; o < K::NFWD; ++o)
        fft_smem<-1>(sm + o * rtile + rr * L1, 1, cfg.pr, rj, ract, tw, TN);
#pragma unroll
      for (int o = 0; o < K::NFWD; ++o) {
        C* S = scr + (size_t)(ri * K::NARR + o) * L + (size_t)j2a * L1;
        for (int e = tid; e < rtile; e += T) {
          const int row = e / L1, k1 = e - row * L1;
          S[e] = cmulc(sm[o * rtile + e], twd(tw, (j2a + row) * k1 * tq));
        }
      }
      __syncthreads();
    }
  }
  // pass C
  C* H = sm + tile;
  for (int k1a = 0; k1a < L1; k1a += w) {
    for (int ri = 0; ri < K::Q; ++ri) {
#pragma unroll
      for (int o = 0; o < K::NFWD; ++o) {
        const C* S = scr + (size_t)(ri * K::NARR + o) * L;
        for (int e = tid; e < tile; e += T) sm[e] = S[(size_t)(e / w) * L1 + k1a + e % w];
        __syncthreads();
        fft_smem<-1>(sm + cc, w, cfg.pc, ci, cact, tw, TN);
        for (int e = tid; e < tile; e += T) {
          const int k = k1a + e % w + L1 * (e / w);
          if (k < m) {
            C v = K::contrib(o, sm[e], k, ri, m, tw);
            H[o * tile + e] = ri ? cadd(H[o * tile + e], v) : v;
          }
        }
        __syncthreads();
      }
    }
#pragma unroll
    for (int o = 0; o < K::NFWD; ++o)
      for (int e = tid; e < tile; e += T) {
        const int k = k1a + e % w + L1 * (e / w);
        if (k < m) out[o][k] = K::finish(o, H[o * tile + e], k, m);
      }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// the kernel: items from a static list (grid-stride) or a persistent queue
// ---------------------------------------------------------------------------
template <int KIND, class C>
__global__ void __launch_bounds__(kThreads) conv1d_kernel(ConvArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ CfgDev s_cfg;
  __shared__ int s_item[3];
  C* sm = reinterpret_cast<C*>(smem_raw);
  int it = blockIdx.x;
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
    const int first = s_item[1], count = s_item[2];
    if (s_cfg.level == 1) {
      conv_level1<KIND, C>(a, s_cfg, first, count, sm);
    } else {
      conv_level2<KIND, C>(a, s_cfg, first, sm, (C*)(a.scratch + (size_t)blockIdx.x * a.slot_bytes));
    }
    if (!a.persistent) it += gridDim.x;
  }
}

}  // namespace dc

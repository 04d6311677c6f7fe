// Persistent task-queue kernel of the fixed-shape engine (compiled once per
// precision; one instantiation per kind of convolution: binary complex,
// centered Hermitian, ternary, Hermitian gradient rows) and its host-side
// planner.
//
// The queue holds level-1 tasks (a group of same-size instances wholly in
// shared memory) and the three pass tasks of every level-2 instance (column
// tiles of pass A, row groups of pass B, column tiles of pass C; fixed.cuh).
// Blocks take tasks in queue order from an atomic counter (each block
// holds the index of its next task while it runs the current one).  A pass task
// first waits until the pass it reads from is complete, which only tasks
// earlier in the queue can bring about.  The earliest unfinished task waits
// on nothing, and the block holding it either runs it or runs an earlier
// task, which is finished by the same argument, so the queue always drains.  Every wait is bounded: past the limit the block records
// DC_ERR_TIMEOUT in the status word and stops.
//
// Level-2 instances are processed in batches whose passes are staggered in
// the queue (A of batch k, B of batch k-1, C of batch k-2, ...), so a pass
// rarely waits; the scratch of a batch is one of four regions that stay
// in L2, and a batch reuses its region after the batch four earlier has
// finished pass C.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include "fixed.cuh"
#include "fixed.h"
#include "launch.h"

namespace dc {
namespace fx {
namespace DC_FX_P {

// Drops a 128-byte line of dead scratch from L2 without writing it back to
// HBM (the data were read for the last time; the next user overwrites
// them).  Without it L2 evicts the dead lines to DRAM, more than doubling
// the kernel's write traffic.
__device__ __forceinline__ void discard_l2(const void* p) {
  asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

// asynchronous 16-byte global-to-shared copies (L2 only), their commit and wait
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
// one element (8 or 16 bytes) global-to-shared, asynchronously
__device__ __forceinline__ void cp_async_elem(C* dst, const C* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(C) == 16) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// size codes: 2^6..2^16, 3*2^5..3*2^14, 5*2^4..5*2^13
__host__ __device__ constexpr int size_of_code(int c) {
  return c < 11 ? (64 << c) : (c < 21 ? (96 << (c - 11)) : (80 << (c - 21)));
}

__host__ __device__ constexpr int ceil_log2(int x) {
  int l = 0;
  while ((1 << l) < x) ++l;
  return l;
}
// split of the root table of zeta_TN into lo (2^sh entries) and hi
__host__ __device__ constexpr int roots_sh(int TN) { return (ceil_log2(TN) + 1) / 2; }
__host__ __device__ constexpr int roots_count(int TN) {
  return (1 << roots_sh(TN)) + (TN + (1 << roots_sh(TN)) - 1) / (1 << roots_sh(TN));
}

constexpr int kBlocksPerSM = kDouble ? 1 : 2;
// kinds whose kernel carries variant 1 of the two-level splits: FP32 binary
// complex (the batched workload); the others run variant 0 only
__host__ __device__ constexpr bool kVariantKind(int mode) { return !kDouble && mode == MODE_COMPLEX; }
// size codes of the two-level sizes (8192 .. 65536, 12288 .. 49152, 10240 .. 40960)
__host__ __device__ constexpr bool two_level_code(int c) { return (c >= 7 && c <= 10) || (c >= 18 && c <= 20) || c >= 28; }

// Shape of size M in variant V (the two-level split, fixed.cuh; one-level
// sizes have variant 0 only)
template <int M, int V = 0> struct Shape {
  static constexpr bool l1 = is_level1(M);
  // level 1
  static constexpr int E = family_E(M);
  static constexpr int T = M / E;
  static constexpr int G = l1 ? kThreads / T : 0;
  // level 2 (placeholders for level-1 sizes)
  static constexpr int L2 = l1 ? 128 : l2_cols(M, V);
  static constexpr int L1 = l1 ? 128 : M / L2;
  static constexpr int W = l1 ? col_width(16384) : col_width(M, V);
  // rows: E = 12 for the 3 * 2^a family (24 elements per thread spill in
  // the row pass), else the family's E
  static constexpr int E1 = odd_part(L1) == 3 ? 12 : family_E(L1);
  static constexpr int T1 = L1 / E1;
  static constexpr int GR = kThreads / T1;
  static constexpr int nA = L1 / W;
  static constexpr int nB = 2 * L2 / GR;
  static constexpr int nBh = 3 * L2 / GR;   // centered Hermitian: three residues, one packed row each
  static constexpr int EC = l1 ? 16 : col_E(M, V);
  static_assert(l1 || (L1 % W == 0 && (2 * L2) % GR == 0 && (3 * L2) % GR == 0 && L1 * L2 == M),
                "level-2 tiling must be exact");
  static_assert(!l1 || kThreads % T == 0, "level-1 groups must tile the block");
  static constexpr int CB = (int)sizeof(C);
  // level 2: the row groups of pass B, or two column tiles (the transform
  // buffer and the prefetched g tile of pass A)
  static constexpr int smem = l1 ? G * group_stride(M, T) * CB
                                 : (GR * group_stride(L1, T1) * CB > 2 * W * L2 * CB ? GR * group_stride(L1, T1) * CB
                                                                                       : 2 * W * L2 * CB);
  // Root tables: kRootsMax entries at the start of shared memory, enough
  // for zeta_{2m} of every size and zeta_{3m} of the level-1 sizes.  The
  // high half of the zeta_{3m} tables of the Hermitian level-2 sizes goes
  // behind the task data instead.
  static constexpr int herm_roots = roots_count(3 * M);
  static constexpr int herm_lo = 1 << roots_sh(3 * M);
  static constexpr bool herm_behind = !l1 && herm_roots > kRootsMax;
  static constexpr int herm_off = kRootsMax * CB + (smem + 15) / 16 * 16;   // bytes from the start
  static constexpr int base = kRootsMax * CB + smem + (herm_behind ? 16 + (herm_roots - herm_lo) * CB : 0);
  // Stage-twiddle tables (fixed.cuh), behind everything else: those of the
  // rows (L1, E1), then those of the columns (L2, EC) unless the two
  // transforms are the same; none for one-level sizes.
  static constexpr bool tab_same = !l1 && L1 == L2 && E1 == EC;
  static constexpr int tab_col = (l1 || tab_same) ? 0 : StageTab<L1, E1>::lay.total;
  static constexpr int tab_entries =
      l1 ? 0 : tab_col + (tab_same ? StageTab<L1, E1>::lay.total : StageTab<L2, EC>::lay.total);
  static constexpr int tab_off = (base + 15) / 16 * 16;   // bytes from the start
  static constexpr int total = tab_off + tab_entries * CB;
  static_assert(herm_lo <= kRootsMax, "low root table fits its reservation");
  static_assert(roots_count(2 * M) <= kRootsMax && (!l1 || herm_roots <= kRootsMax), "root tables fit");
  static_assert(!l1 || roots_count(4 * M) <= kRootsMax, "the four-residue ternary tables fit");
  // FP32: two blocks per SM, FP64: one (228 KB per SM less 1 KB reserved per
  // block and the static shared variables)
  static_assert(total <= (233472 - kBlocksPerSM * 1024) / kBlocksPerSM - 64, "the blocks fit on an SM");
};

// ---------------------------------------------------------------------------
// device side
// ---------------------------------------------------------------------------

// One-level transforms form their stage twiddles by products; the row and
// column transforms of two-level sizes read their stage tables, which sit
// at a fixed place of the block's dynamic shared memory (so their address
// is a constant, not a register held across the task).
extern __shared__ __align__(16) unsigned char fx_smem[];
template <int M, int V> __device__ __forceinline__ TabRoots row_roots(const Roots<C>& r) {
  return TabRoots{r, (const C*)(fx_smem + Shape<M, V>::tab_off)};
}
template <int M, int V> __device__ __forceinline__ TabRoots col_roots(const Roots<C>& r) {
  return TabRoots{r, (const C*)(fx_smem + Shape<M, V>::tab_off) + Shape<M, V>::tab_col};
}
template <int M, int V> __device__ __forceinline__ void gen_size_tabs(C* st) {
  using S = Shape<M, V>;
  if constexpr (!S::l1) {
    gen_stage_tabs<S::L1, S::E1>(st);
    if constexpr (!S::tab_same) gen_stage_tabs<S::L2, S::EC>(st + S::tab_col);
  }
}


// Residue r of a centered Hermitian convolution (Sec. 2.3, N = 3m), in a
// form without branches on r or k, so that the loads of all E elements of
// a thread can be issued together.  The packed input of f and g at k is
// zeta_{3m}^{rk} (P_k + zeta_3^{-r} Q_k) with P_k = f_k + i g_k and
// Q_k = conj f_{m-k} + i conj g_{m-k} (Eqs. (2.4)-(2.5) with Hermitian
// symmetry); at k = 0 it is Re f_0 + i Re g_0.  For r = 0 both factors are
// 1 (the table lookup at index 0).  The output factor is zeta_{3m}^{-rk}
// (Eq. (2.7)).
struct HermTerms {
  int r;
  C z3;   // zeta_3^{-r}, 1 for r = 0
  __device__ __forceinline__ explicit HermTerms(int r_) : r(r_) {
    z3.x = r_ ? (Real)-0.5 : (Real)1;
    z3.y = (Real)(-r_) * (Real)0.86602540378443864676;
  }
  // zeta_{3m}^{s r k}
  __device__ __forceinline__ C tw(int x, const Roots<C>& rt, int s) const {
    C t = rt.at(r ? x : 0);
    if (r * s < 0) t.y = -t.y;
    return t;
  }
  template <int M>
  __device__ __forceinline__ C packed(const C* f, const C* g, int x, const Roots<C>& rt) const {
    const int mx = x ? M - x : 0;
    const C fk = __ldg(f + x), gk = __ldg(g + x), fm = __ldg(f + mx), gm = __ldg(g + mx);
    C P, Q;
    P.x = fk.x - gk.y;
    P.y = fk.y + gk.x;
    Q.x = fm.x + gm.y;
    Q.y = gm.x - fm.y;
    C v = cmul(cadd(P, cmul(Q, z3)), tw(x, rt, 1));
    if (x == 0) {
      v.x = fk.x;
      v.y = gk.x;
    }
    return v;
  }
  template <int M>
  __device__ __forceinline__ C single(const C* u, int x, const Roots<C>& rt) const {
    const int mx = x ? M - x : 0;
    const C p = __ldg(u + x);
    C q = __ldg(u + mx);
    q.y = -q.y;
    C v = cmul(cadd(p, cmul(q, z3)), tw(x, rt, 1));
    if (x == 0) {
      v.x = p.x;
      v.y = 0;
    }
    return v;
  }
  __device__ __forceinline__ C out(C v, int x, const Roots<C>& rt) const { return cmul(v, tw(x, rt, -1)); }
};

// Residue r = 0..3 of a centered Hermitian ternary convolution taken as four
// m-point residues of the N = 4m padding (Sec. 4.1's padding; the fold of
// Sec. 2.2 with zeta_4 for zeta_3): the input at k > 0 is
// zeta_{4m}^{rk} (U_k + zeta_4^{-r} U_{k-m}), U_{k-m} = conj U_{m-k}, and at
// k = 0 it is U_0 (U_{-m} = 0); the output factor is zeta_{4m}^{-rk}.
struct Tern4Terms {
  int r;
  C z4;   // zeta_4^{-r} = (-i)^r
  __device__ __forceinline__ explicit Tern4Terms(int r_) : r(r_) {
    z4.x = r_ == 0 ? (Real)1 : (r_ == 2 ? (Real)-1 : (Real)0);
    z4.y = r_ == 1 ? (Real)-1 : (r_ == 3 ? (Real)1 : (Real)0);
  }
  // zeta_{4m}^{s r k} (r k < 3m: inside the table of zeta_{4m})
  __device__ __forceinline__ C tw(int x, const Roots<C>& rt, int s) const {
    C t = rt.at(r * x);
    if (s < 0) t.y = -t.y;
    return t;
  }
  // f + i g packed (both backward transforms are real)
  template <int M>
  __device__ __forceinline__ C packed(const C* f, const C* g, int x, const Roots<C>& rt) const {
    const int mx = x ? M - x : 0;
    const C fk = __ldg(f + x), gk = __ldg(g + x), fm = __ldg(f + mx), gm = __ldg(g + mx);
    C P, Q;
    P.x = fk.x - gk.y;
    P.y = fk.y + gk.x;
    Q.x = fm.x + gm.y;
    Q.y = gm.x - fm.y;
    C v = cmul(cadd(P, cmul(Q, z4)), tw(x, rt, 1));
    if (x == 0) {
      v.x = fk.x;
      v.y = gk.x;
    }
    return v;
  }
  template <int M>
  __device__ __forceinline__ C single(const C* u, int x, const Roots<C>& rt) const {
    const int mx = x ? M - x : 0;
    const C p = __ldg(u + x);
    C q = __ldg(u + mx);
    q.y = -q.y;
    C v = cmul(cadd(p, cmul(q, z4)), tw(x, rt, 1));
    if (x == 0) {
      v.x = p.x;
      v.y = 0;
    }
    return v;
  }
  __device__ __forceinline__ C out(C v, int x, const Roots<C>& rt) const { return cmul(v, tw(x, rt, -1)); }
};

// level 1: residue R of `count` instances of size M, one thread group each.
// One function per residue: inlining both lets the compiler share index
// arithmetic across them, which costs registers and spills.
template <int M, int R>
__device__ __noinline__ void l1_residue(const FxArgs* a, int first, int count, C* sm, Roots<C> rt) {
  using S = Shape<M>;
  constexpr int E = S::E, T = S::T, PL = padded(M), GS = group_stride(M, T), TN = 2 * M;
  const int gi = threadIdx.x / T, i = threadIdx.x % T;
  const bool act = gi < count;
  const int64_t off = act ? a->off[a->order[first + gi]] : 0;
  const C* f = (const C*)a->f + off;
  const C* g = (const C*)a->g + off;
  C* h = (C*)a->h + off;
  // Residue 0's partial output: in h itself, or, when h is f or g (in-place
  // calls), in a region of the workspace, so that h is written only at
  // residue 1, after every read of f and g.
  C* hp = a->in_place ? (C*)a->tmp + (act ? a->l1tmp[a->order[first + gi]] : 0) : h;
  C* A = sm + gi * GS;
  C* B = A + PL;
  const Real sc = (Real)1 / (Real)(2 * M);
  const GroupSync<T> sync{1 + gi};
  // groups past `count` transform zeros and store nothing: the stages
  // themselves carry no condition
  C zero;
  zero.x = 0;
  zero.y = 0;
  if constexpr (R == 0) {
    // residue 0 (Eq. (2.1) with r = 0): partial output
    conv_residue<M, E, TN>(
        i, true, A, B, rt, [&](int x, int arr, int) { return act ? __ldg((arr ? g : f) + x) : zero; },
        [&](int x, int, C v) {
          if (act) hp[x] = cscale(v, sc);
        },
        sync);
  } else {
    // residue 1: inputs times zeta_{2m}^k, output times zeta_{2m}^{-k}
    // (Eq. (2.2)).  The last forward stage leaves register e at the position
    // the first backward stage loaded into it, so one lookup per element
    // serves f, g and the output.
    C tw[E];
    auto ld = [&](int x, int arr, int e) {
      if (arr == 0) tw[e] = rt.at(x);
      return act ? cmul(__ldg((arr ? g : f) + x), tw[e]) : zero;
    };
    if constexpr (E <= 20) {
      conv_residue<M, E, TN>(
          i, true, A, B, rt, ld,
          [&](int x, int e, C v) {
            if (act) h[x] = cadd(hp[x], cscale(cmulc(v, tw[e]), sc));
          },
          sync);
    } else {
      // E = 24: a second lookup is cheaper than 24 registers held through
      // the whole residue
      conv_residue<M, E, TN>(
          i, true, A, B, rt, ld,
          [&](int x, int, C v) {
            if (act) h[x] = cadd(hp[x], cscale(cmulc(v, rt.at(x)), sc));
          },
          sync);
    }
  }
}

// level 1, centered Hermitian (Sec. 2.3, N = 3m): residue ri (r = ri - 1)
// of `count` instances.  The input of residue r is
// w_{k,r} = zeta_{3m}^{rk} (U_k + zeta_3^{-r} conj U_{m-k}) for k > 0 and
// Re U_0 at k = 0 (Eqs. (2.4)-(2.5) with Hermitian symmetry, U_0 taken
// real), packed as w^f + i w^g; the output adds zeta_{3m}^{-rk} S_r(k) / 3m
// (Eq. (2.7)) for k < m.
template <int M>
__device__ __noinline__ void l1_herm_residue(const FxArgs* a, int ri, int first, int count, C* sm, Roots<C> rt) {
  using S = Shape<M>;
  constexpr int E = S::E, T = S::T, PL = padded(M), GS = group_stride(M, T), TN = 3 * M;
  const int gi = threadIdx.x / T, i = threadIdx.x % T;
  const bool act = gi < count;
  const int64_t off = act ? a->off[a->order[first + gi]] : 0;
  const C* f = (const C*)a->f + off;
  const C* g = (const C*)a->g + off;
  C* h = (C*)a->h + off;
  C* A = sm + gi * GS;
  // The transform uses the group's first array only; the second holds the
  // sum over the residues.  Output k of a thread sits at the same position
  // in every residue, so the sum needs no barrier, and h is written once,
  // at the last residue (after every read of f and g, so h may be f or g).
  const Contig acc{A + PL};
  const Real sc = (Real)1 / (Real)(3 * M);
  const GroupSync<T> sync{1 + gi};
  const HermTerms ht(ri - 1);
  conv1_residue<M, E, TN>(
      i, A, rt,
      [&](int x, int) {
        C v = ht.packed<M>(f, g, x, rt);
        if (!act) v.x = v.y = 0;
        return v;
      },
      [&](int x, int, C v) {
        v = cscale(ht.out(v, x, rt), sc);
        C prev;
        prev.x = prev.y = 0;
        if (ri) prev = acc[x];
        v = cadd(prev, v);
        if (ri < 2) acc[x] = v;
        else if (act) h[x] = v;
      },
      sync);
}

// level 1, rows of a centered Hermitian gradient: residue ri (r = ri - 1)
// of `count` instances.  Inputs W, f, g (in f, g, e); outputs conv(W, g)
// (h) and conv(W, f) (h2), each Eq. (2.7) with the residue inputs w_{k,r}
// of l1_herm_residue.  W is transformed alone and f, g packed.  In-place
// calls keep both partial outputs in two slots of the workspace.
template <int M>
__device__ __noinline__ void l1_pair_residue(const FxArgs* a, int ri, int first, int count, C* sm, Roots<C> rt) {
  using S = Shape<M>;
  constexpr int E = S::E, T = S::T, PL = padded(M), GS = group_stride(M, T), TN = 3 * M;
  const int gi = threadIdx.x / T, i = threadIdx.x % T;
  const bool act = gi < count;
  const int64_t off = act ? a->off[a->order[first + gi]] : 0;
  const C* w = (const C*)a->f + off;
  const C* f = (const C*)a->g + off;
  const C* g = (const C*)a->e + off;
  C* h0 = (C*)a->h + off;
  C* h1 = (C*)a->h2 + off;
  C* p0 = a->in_place ? (C*)a->tmp + (act ? a->l1tmp[a->order[first + gi]] : 0) : h0;
  C* p1 = a->in_place ? p0 + M : h1;
  C* A = sm + gi * GS;
  const Real sc = (Real)1 / (Real)(3 * M);
  const GroupSync<T> sync{1 + gi};
  const HermTerms ht(ri - 1);
  conv_pair_residue<M, E, TN>(
      i, A, A + PL, rt,
      [&](int x, int arr, int) {
        C v = arr == 0 ? ht.single<M>(w, x, rt) : ht.packed<M>(f, g, x, rt);
        if (!act) v.x = v.y = 0;
        return v;
      },
      [&](int x, int, C v, int o) {
        if (!act) return;
        v = cscale(ht.out(v, x, rt), sc);
        C* p = o ? p1 : p0;
        C prev;
        prev.x = prev.y = 0;
        if (ri) prev = p[x];
        (ri == 2 ? (o ? h1 : h0) : p)[x] = cadd(prev, v);
      },
      sync);
}

// product of the dot product of two centered Hermitian pairs: the first
// array holds u^{f1} + i u^{g1}, the second u^{f2} + i u^{g2} (all four
// real), and the sum of the two real products is real
struct HDot2Prod {
  __device__ __forceinline__ C operator()(C a, C b) const {
    C p;
    p.x = a.x * a.y + b.x * b.y;
    p.y = 0;
    return p;
  }
};

// level 1, dot product of two centered Hermitian pairs (Sec. 3, arrays of
// vectors; Sec. 2.3 per pair): residue ri (r = ri - 1) of `count`
// instances.  The group's two arrays take the packed inputs
// w^{f1} + i w^{g1} and w^{f2} + i w^{g2}; both backward transforms, the
// summed real product, one forward transform; the output adds
// zeta_{3m}^{-rk} S_r(k) / 3m.  The residue sum is kept in h, or, for
// in-place calls (h one of the inputs), in a workspace slot, and h is
// written at the last residue.
template <int M>
__device__ __noinline__ void l1_hdot2_residue(const FxArgs* a, int ri, int first, int count, C* sm, Roots<C> rt) {
  using S = Shape<M>;
  constexpr int E = S::E, T = S::T, PL = padded(M), GS = group_stride(M, T), TN = 3 * M;
  const int gi = threadIdx.x / T, i = threadIdx.x % T;
  const bool act = gi < count;
  const int64_t off = act ? a->off[a->order[first + gi]] : 0;
  const C* f1 = (const C*)a->f + off;
  const C* g1 = (const C*)a->g + off;
  const C* f2 = (const C*)a->e + off;
  const C* g2 = (const C*)a->e2 + off;
  C* h = (C*)a->h + off;
  C* p = a->in_place ? (C*)a->tmp + (act ? a->l1tmp[a->order[first + gi]] : 0) : h;
  C* A = sm + gi * GS;
  const Real sc = (Real)1 / (Real)(3 * M);
  const GroupSync<T> sync{1 + gi};
  const HermTerms ht(ri - 1);
  conv_residue<M, E, TN>(
      i, true, A, A + PL, rt,
      [&](int x, int arr, int) {
        C v = arr ? ht.packed<M>(f2, g2, x, rt) : ht.packed<M>(f1, g1, x, rt);
        if (!act) v.x = v.y = 0;
        return v;
      },
      [&](int x, int, C v) {
        if (!act) return;
        v = cscale(ht.out(v, x, rt), sc);
        if (ri == 0) p[x] = v;
        else if (ri == 1) p[x] = cadd(p[x], v);
        else h[x] = cadd(p[x], v);
      },
      sync, HDot2Prod{});
}

// Ternary product of the four-residue form: the first array holds
// u^f + i u^g, the second u^e (all real); the triple product is real.
struct Tern4Prod {
  __device__ __forceinline__ C operator()(C a, C b) const {
    C p;
    p.x = a.x * a.y * b.x;
    p.y = 0;
    return p;
  }
};

// level 1, centered Hermitian ternary convolution of length m = M as four
// m-point residues (Tern4Terms): residue ri of `count` instances.  The
// group's two arrays take the packed f + i g and e; both backward
// transforms, the triple product, one forward transform; the output adds
// zeta_{4m}^{-rk} S_r(k) / 4m, k < m.  The residue sum is kept in h, or,
// for in-place calls, in a workspace slot, and h is written at the last
// residue.
template <int M>
__device__ __noinline__ void l1_tern4_residue(const FxArgs* a, int ri, int first, int count, C* sm, Roots<C> rt) {
  using S = Shape<M>;
  constexpr int E = S::E, T = S::T, PL = padded(M), GS = group_stride(M, T), TN = 4 * M;
  const int gi = threadIdx.x / T, i = threadIdx.x % T;
  const bool act = gi < count;
  const int64_t off = act ? a->off[a->order[first + gi]] : 0;
  const C* f = (const C*)a->f + off;
  const C* g = (const C*)a->g + off;
  const C* e = (const C*)a->e + off;
  C* h = (C*)a->h + off;
  C* p = a->in_place ? (C*)a->tmp + (act ? a->l1tmp[a->order[first + gi]] : 0) : h;
  C* A = sm + gi * GS;
  const Real sc = (Real)1 / (Real)(4 * M);
  const GroupSync<T> sync{1 + gi};
  const Tern4Terms tt(ri);
  conv_residue<M, E, TN>(
      i, true, A, A + PL, rt,
      [&](int x, int arr, int) {
        C v = arr ? tt.single<M>(e, x, rt) : tt.packed<M>(f, g, x, rt);
        if (!act) v.x = v.y = 0;
        return v;
      },
      [&](int x, int, C v) {
        if (!act) return;
        v = cscale(tt.out(v, x, rt), sc);
        if (ri == 0) p[x] = v;
        else if (ri < 3) p[x] = cadd(p[x], v);
        else h[x] = cadd(p[x], v);
      },
      sync, Tern4Prod{});
}

// pass A: column tile `tile` of level-2 instance l.  Each pass is its own
// function so that registers are allocated per pass.
template <int M, int V>
__device__ __noinline__ void run_A(const FxArgs* a, int l, int tile, C* sm, Roots<C> rt) {
  using S = Shape<M, V>;
  constexpr int L1 = S::L1, L2 = S::L2, W = S::W, E = S::EC, TN = 2 * M;
  using K = Stage<L2, E, 0, false>;
  const int c = threadIdx.x % W, i = threadIdx.x / W;
  const int k1 = tile * W + c;
  const L2Inst in = a->l2[l];
  C* scr = (C*)a->scratch + in.scr;
  // residue-1 input twiddles zeta_{2m}^{k1 + L1 k2}, shared by f and g
  C tw[E];
#pragma unroll
  for (int b = 0; b < K::NB; ++b)
#pragma unroll
    for (int q = 0; q < K::R; ++q) tw[b * K::R + q] = rt.at(k1 + L1 * pos<L2, E, 0, false>(i, b, q));
  // g's column tile comes into shared memory, behind the transform buffer,
  // while f's columns are transformed (16-byte copies; instance offsets and
  // tile starts are multiples of 16 elements)
  C* gt = sm + W * L2;
  {
    constexpr int CPR = W * (int)sizeof(C) / 16;   // 16-byte chunks per tile row
    const char* gsrc = (const char*)((const C*)a->g + in.off + (size_t)tile * W);
    for (int ch = threadIdx.x; ch < L2 * CPR; ch += kThreads) {
      const int row = ch / CPR, col = ch % CPR;
      cp_async16((char*)gt + ((size_t)row * W * sizeof(C) + (size_t)col * 16),
                 gsrc + ((size_t)row * L1 * sizeof(C) + (size_t)col * 16));
    }
    cp_async_commit();
  }
#pragma unroll 1
  for (int arr = 0; arr < 2; ++arr) {
    C raw[E];
    if (arr == 0) {
      const C* x = (const C*)a->f + in.off + k1;
#pragma unroll
      for (int b = 0; b < K::NB; ++b)
#pragma unroll
        for (int q = 0; q < K::R; ++q) raw[b * K::R + q] = __ldg(x + L1 * pos<L2, E, 0, false>(i, b, q));
    } else {
      cp_async_wait_all();
      __syncthreads();
#pragma unroll
      for (int b = 0; b < K::NB; ++b)
#pragma unroll
        for (int q = 0; q < K::R; ++q) raw[b * K::R + q] = gt[pos<L2, E, 0, false>(i, b, q) * W + c];
    }
#pragma unroll 1
    for (int r = 0; r < 2; ++r) {
      C v[E];
#pragma unroll
      for (int e = 0; e < E; ++e) v[e] = r ? cmul(raw[e], tw[e]) : raw[e];
      // S[j2][k1]; the factor zeta_m^{j2 k1} is applied in pass B
      C* dst = scr + (size_t)(2 * r + arr) * M + k1;
      column<L2, E, W, TN, false>(v, i, sm + c, col_roots<M, V>(rt), [&](int j2, int, C y) { __stcg(dst + (size_t)j2 * L1, y); });
      __syncthreads();
    }
  }
}

// pass A of a centered Hermitian ternary convolution (Sec. 4.2, N = 4m) on
// the M = 2m point sub-transforms: column tile `tile` of level-2 instance
// l.  Residue r = 0, 1 transforms V_k = zeta_{4m}^{rk} U_k (k < m, U_0 real),
// V_m = 0, V_k = conj V_{2m-k} (k > m), of f + i g (first array) and of e
// (second).  With B_k = U_k (k < m), conj U_{2m-k} (k > m), V_k equals
// zeta_{4m}^{rk} B_k times (-1)^r above m, since zeta_{4m}^{2m} = -1; the
// residue-1 factor below carries that sign.
template <int M, int V>
__device__ __noinline__ void run_A_tern(const FxArgs* a, int l, int tile, C* sm, Roots<C> rt) {
  using S = Shape<M, V>;
  constexpr int L1 = S::L1, L2 = S::L2, W = S::W, E = S::EC, TN = 2 * M, MH = M / 2;
  using K = Stage<L2, E, 0, false>;
  const int c = threadIdx.x % W, i = threadIdx.x / W;
  const int k1 = tile * W + c;
  const L2Inst in = a->l2[l];
  C* scr = (C*)a->scratch + in.scr;
  C tw[E];
#pragma unroll
  for (int b = 0; b < K::NB; ++b)
#pragma unroll
    for (int q = 0; q < K::R; ++q) {
      const int k = k1 + L1 * pos<L2, E, 0, false>(i, b, q);
      C t = rt.at(k);
      if (k > MH) {
        t.x = -t.x;
        t.y = -t.y;
      }
      tw[b * K::R + q] = t;
    }
#pragma unroll 1
  for (int arr = 0; arr < 2; ++arr) {
    const C* u = (const C*)(arr ? a->e : a->f) + in.off;
    const C* ug = (const C*)a->g + in.off;
    C raw[E];
#pragma unroll
    for (int b = 0; b < K::NB; ++b)
#pragma unroll
      for (int q = 0; q < K::R; ++q) {
        const int k = k1 + L1 * pos<L2, E, 0, false>(i, b, q);
        const bool up = k > MH;
        const int kk = k < MH ? k : (up ? M - k : 0);
        C x = __ldg(u + kk);
        C y;   // B_k of the second array packed as the imaginary part
        if (arr == 0) {
          const C gv = __ldg(ug + kk);
          if (k == 0) {
            y.x = x.x;
            y.y = gv.x;
          } else if (up) {   // conj f + i conj g
            y.x = x.x + gv.y;
            y.y = gv.x - x.y;
          } else {           // f + i g
            y.x = x.x - gv.y;
            y.y = x.y + gv.x;
          }
        } else {
          y.x = x.x;
          y.y = k == 0 ? (Real)0 : (up ? -x.y : x.y);
        }
        if (k == MH) {
          y.x = 0;
          y.y = 0;
        }
        raw[b * K::R + q] = y;
      }
#pragma unroll 1
    for (int r = 0; r < 2; ++r) {
      C v[E];
#pragma unroll
      for (int e = 0; e < E; ++e) v[e] = r ? cmul(raw[e], tw[e]) : raw[e];
      C* dst = scr + (size_t)(2 * r + arr) * M + k1;
      column<L2, E, W, TN, false>(v, i, sm + c, col_roots<M, V>(rt), [&](int j2, int, C y) { __stcg(dst + (size_t)j2 * L1, y); });
      __syncthreads();
    }
  }
}

// Ternary product (Sec. 4.2): the first array holds u^f + i u^g, the second
// u^e (both real), their triple product is real.
struct TernProd {
  __device__ __forceinline__ C operator()(C a, C b) const {
    C p;
    p.x = a.x * a.y * b.x;
    p.y = 0;
    return p;
  }
};

// pass B: row group `unit` (rows (r, j2), r = row / L2) of level-2 instance
// l; TERN: the ternary product of a ternary convolution's sub-transforms
template <int M, int V, bool TERN>
__device__ __noinline__ void run_B(const FxArgs* a, int l, int unit, C* sm, Roots<C> rt) {
  using S = Shape<M, V>;
  constexpr int L1 = S::L1, L2 = S::L2, E1 = S::E1, T1 = S::T1, GR = S::GR, PL = padded(L1),
                GS = group_stride(L1, T1), TN = 2 * M;
  const int gi = threadIdx.x / T1, i = threadIdx.x % T1;
  const int row = unit * GR + gi;
  const int r = row / L2, j2 = row % L2;
  C* scr = (C*)a->scratch + a->l2[l].scr;
  C* sf = scr + (size_t)(2 * r) * M + (size_t)j2 * L1;
  const C* sg = scr + (size_t)(2 * r + 1) * M + (size_t)j2 * L1;
  C* A = sm + gi * GS;
  C* B = A + PL;
  // inputs times zeta_m^{j2 k1} (one lookup for f, g and the output, whose
  // register e sits at the same position), output times zeta_m^{-j2 k1}
  const GroupSync<T1> sync{1 + gi};
  static_assert(E1 <= 20, "rows hold their twiddles in registers");
  C tw[E1];
  conv_residue<L1, E1, TN>(
      i, true, A, B, row_roots<M, V>(rt),
      [&](int x, int arr, int e) {
        if (arr == 0) tw[e] = rt.at(2 * j2 * x);
        return cmul(__ldcg((arr ? sg : (const C*)sf) + x), tw[e]);
      },
      [&](int x, int e, C v) { __stcg(sf + x, cmulc(v, tw[e])); }, sync,
      typename std::conditional<TERN, TernProd, CProd>::type{});
  // the g row was read for the last time (every thread of the group loaded
  // its part before the group's first barrier)
  for (int ln = i; ln < L1 * (int)sizeof(C) / 128; ln += T1) discard_l2((const char*)sg + ln * 128);
}

// pass C: column tile `tile` of level-2 instance l, both residues, output;
// TERN: only the outputs k < M / 2 (a ternary convolution's length)
template <int M, int V, bool TERN>
__device__ __noinline__ void run_C(const FxArgs* a, int l, int tile, C* sm, Roots<C> rt) {
  using S = Shape<M, V>;
  constexpr int L1 = S::L1, L2 = S::L2, W = S::W, E = S::EC, TN = 2 * M;
  using K = Stage<L2, E, 0, true>;
  const int c = threadIdx.x % W, i = threadIdx.x / W;
  const int k1 = tile * W + c;
  const L2Inst in = a->l2[l];
  const C* scr = (const C*)a->scratch + in.scr;
  C* h = (C*)a->h + in.off + k1;
  const Real sc = (Real)1 / (Real)(2 * M);
  C y0[E];
  C vin[2][E];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const C* src = scr + (size_t)(2 * r) * M + k1;
#pragma unroll
    for (int b = 0; b < K::NB; ++b)
#pragma unroll
      for (int q = 0; q < K::R; ++q) vin[r][b * K::R + q] = __ldcg(src + (size_t)L1 * pos<L2, E, 0, true>(i, b, q));
  }
  column<L2, E, W, TN, true>(vin[0], i, sm + c, col_roots<M, V>(rt), [&](int, int e, C y) { y0[e] = y; });
  __syncthreads();
  column<L2, E, W, TN, true>(vin[1], i, sm + c, col_roots<M, V>(rt), [&](int k2, int e, C y) {
    const int k = k1 + L1 * k2;
    if (!TERN || 2 * k2 < L2) h[(size_t)L1 * k2] = cscale(cadd(y0[e], cmulc(y, rt.at(k))), sc);
  });
  // both residues' product columns of the tile were read for the last time
  __syncthreads();
  constexpr int LPR = W * (int)sizeof(C) / 128;   // 128-byte lines per tile row
  for (int ln = threadIdx.x; ln < 2 * L2 * LPR; ln += kThreads) {
    const int rr = ln / (L2 * LPR), rest = ln % (L2 * LPR);
    const C* row = scr + (size_t)(2 * rr) * M + (size_t)(rest / LPR) * L1 + (size_t)tile * W;
    discard_l2((const char*)row + (rest % LPR) * 128);
  }
}

// Level 2 of a centered Hermitian convolution (Sec. 2.3, N = 3m): the three
// residues r = -1, 0, 1 each hold one packed array w^f + i w^g (both
// backward transforms are real), in scratch arrays ri = r + 1.
//
// pass A: column tile `tile` of level-2 instance l.  With P_k = f_k + i g_k
// and Q_k = conj f_{m-k} + i conj g_{m-k}, residue r's packed input is
// zeta_{3m}^{rk} (P_k + zeta_3^{-r} Q_k) (Eqs. (2.4)-(2.5) with Hermitian
// symmetry); at k = 0 it is Re f_0 + i Re g_0 for every r.
template <int M, int V>
__device__ __noinline__ void run_A_herm(const FxArgs* a, int l, int tile, C* sm, Roots<C> rt) {
  using S = Shape<M, V>;
  constexpr int L1 = S::L1, L2 = S::L2, W = S::W, E = S::EC, TN = 3 * M;
  using K = Stage<L2, E, 0, false>;
  const int c = threadIdx.x % W, i = threadIdx.x / W;
  const int k1 = tile * W + c;
  const L2Inst in = a->l2[l];
  C* scr = (C*)a->scratch + in.scr;
  const C* f = (const C*)a->f + in.off;
  const C* g = (const C*)a->g + in.off;
  C P[E], Q[E];
#pragma unroll
  for (int b = 0; b < K::NB; ++b)
#pragma unroll
    for (int q = 0; q < K::R; ++q) {
      const int e = b * K::R + q;
      const int k = k1 + L1 * pos<L2, E, 0, false>(i, b, q);
      const int mk = k ? M - k : 0;
      const C fk = __ldg(f + k), gk = __ldg(g + k), fm = __ldg(f + mk), gm = __ldg(g + mk);
      P[e].x = k ? fk.x - gk.y : fk.x;
      P[e].y = k ? fk.y + gk.x : gk.x;
      Q[e].x = k ? fm.x + gm.y : (Real)0;
      Q[e].y = k ? gm.x - fm.y : (Real)0;
    }
#pragma unroll 1
  for (int ri = 0; ri < 3; ++ri) {
    const int r = ri - 1;
    C z3;   // zeta_3^{-r}
    z3.x = (Real)-0.5;
    z3.y = (Real)(-r) * (Real)0.86602540378443864676;
    C v[E];
#pragma unroll
    for (int b = 0; b < K::NB; ++b)
#pragma unroll
      for (int q = 0; q < K::R; ++q) {
        const int e = b * K::R + q;
        C w = r == 0 ? cadd(P[e], Q[e]) : cadd(P[e], cmul(Q[e], z3));
        if (r != 0) {
          const C t = rt.at(k1 + L1 * pos<L2, E, 0, false>(i, b, q));
          w = r > 0 ? cmul(w, t) : cmulc(w, t);
        }
        v[e] = w;
      }
    // S_r[j2][k1]; the factor zeta_m^{j2 k1} is applied in pass B
    C* dst = scr + (size_t)ri * M + k1;
    column<L2, E, W, TN, false>(v, i, sm + c, col_roots<M, V>(rt), [&](int j2, int, C y) { __stcg(dst + (size_t)j2 * L1, y); });
    __syncthreads();
  }
}

// pass B: row group `unit` (rows (ri, j2), ri = row / L2) of level-2
// instance l: times zeta_m^{j2 k1}, backward row transform, the real
// product u^f u^g, forward row transform, times zeta_m^{-j2 k1}, in place
template <int M, int V>
__device__ __noinline__ void run_B_herm(const FxArgs* a, int l, int unit, C* sm, Roots<C> rt) {
  using S = Shape<M, V>;
  constexpr int L1 = S::L1, L2 = S::L2, E1 = S::E1, T1 = S::T1, GR = S::GR, GS = group_stride(L1, T1),
                TN = 3 * M;
  const int gi = threadIdx.x / T1, i = threadIdx.x % T1;
  const int row = unit * GR + gi;
  const int ri = row / L2, j2 = row % L2;
  C* s = (C*)a->scratch + a->l2[l].scr + (size_t)ri * M + (size_t)j2 * L1;
  const GroupSync<T1> sync{1 + gi};
  static_assert(E1 <= 20, "rows hold their twiddles in registers");
  C tw[E1];
  conv1_residue<L1, E1, TN>(
      i, sm + gi * GS, row_roots<M, V>(rt),
      [&](int x, int e) {
        tw[e] = rt.at(3 * j2 * x);
        return cmul(__ldcg(s + x), tw[e]);
      },
      [&](int x, int e, C v) { __stcg(s + x, cmulc(v, tw[e])); }, sync);
}

// pass C: column tile `tile` of level-2 instance l: the forward column
// transforms of the three residues, recombined as
// h_k = sum_r zeta_{3m}^{-rk} S_r(k) / 3m (Eq. (2.7)), k < m
template <int M, int V>
__device__ __noinline__ void run_C_herm(const FxArgs* a, int l, int tile, C* sm, Roots<C> rt) {
  using S = Shape<M, V>;
  constexpr int L1 = S::L1, L2 = S::L2, W = S::W, E = S::EC, TN = 3 * M;
  using K = Stage<L2, E, 0, true>;
  const int c = threadIdx.x % W, i = threadIdx.x / W;
  const int k1 = tile * W + c;
  const L2Inst in = a->l2[l];
  const C* scr = (const C*)a->scratch + in.scr;
  C* h = (C*)a->h + in.off + k1;
  const Real sc = (Real)1 / (Real)(3 * M);
  C acc[E];
#pragma unroll 1
  for (int ri = 0; ri < 3; ++ri) {
    const int r = ri - 1;
    const C* src = scr + (size_t)ri * M + k1;
    C v[E];
#pragma unroll
    for (int b = 0; b < K::NB; ++b)
#pragma unroll
      for (int q = 0; q < K::R; ++q) v[b * K::R + q] = __ldcg(src + (size_t)L1 * pos<L2, E, 0, true>(i, b, q));
    column<L2, E, W, TN, true>(v, i, sm + c, col_roots<M, V>(rt), [&](int k2, int e, C y) {
      if (r != 0) {
        const C t = rt.at(k1 + L1 * k2);
        y = r > 0 ? cmulc(y, t) : cmul(y, t);
      }
      if (ri == 0) acc[e] = y;
      else if (ri == 1) acc[e] = cadd(acc[e], y);
      else h[(size_t)L1 * k2] = cscale(cadd(acc[e], y), sc);
    });
    __syncthreads();
  }
  // the three product columns of the tile were read for the last time
  constexpr int LPR = W * (int)sizeof(C) / 128;   // 128-byte lines per tile row
  for (int ln = threadIdx.x; ln < 3 * L2 * LPR; ln += kThreads) {
    const int rr = ln / (L2 * LPR), rest = ln % (L2 * LPR);
    const C* row = scr + (size_t)rr * M + (size_t)(rest / LPR) * L1 + (size_t)tile * W;
    discard_l2((const char*)row + (rest % LPR) * 128);
  }
}

// One kernel per kind of convolution (MODE_*), so that each kernel's call
// graph (and the registers ptxas gives its functions) holds only its own
// passes.

template <int M, int V, int MODE>
__device__ __noinline__ void run_size(const FxArgs* a, int type, int x, int y, int units, C* sm, Roots<C> rt) {
  if constexpr (Shape<M>::l1) {
    if constexpr (MODE == MODE_HERM) {
#pragma unroll 1
      for (int ri = 0; ri < 3; ++ri) {
        l1_herm_residue<M>(a, ri, x, y, sm, rt);
        __syncthreads();
      }
    } else if constexpr (MODE == MODE_COMPLEX) {
      l1_residue<M, 0>(a, x, y, sm, rt);
      __syncthreads();
      l1_residue<M, 1>(a, x, y, sm, rt);
    } else if constexpr (MODE == MODE_PAIR) {
#pragma unroll 1
      for (int ri = 0; ri < 3; ++ri) {
        l1_pair_residue<M>(a, ri, x, y, sm, rt);
        __syncthreads();
      }
    } else if constexpr (MODE == MODE_HDOT2) {
#pragma unroll 1
      for (int ri = 0; ri < 3; ++ri) {
        l1_hdot2_residue<M>(a, ri, x, y, sm, rt);
        __syncthreads();
      }
    } else if constexpr (MODE == MODE_TERN4) {
#pragma unroll 1
      for (int ri = 0; ri < 4; ++ri) {
        l1_tern4_residue<M>(a, ri, x, y, sm, rt);
        __syncthreads();
      }
    } else {
      // ternary plans hold two-level sizes only (the planner refuses others)
      if (threadIdx.x == 0) record_error(a->hdr, DC_ERR_DEVICE, M);
    }
  } else {
    if constexpr (MODE == MODE_PAIR || MODE == MODE_HDOT2 || MODE == MODE_TERN4) {
      // gradient-pair, dot-product and four-residue ternary plans hold
      // one-level sizes only (the planner refuses others)
      if (threadIdx.x == 0) record_error(a->hdr, DC_ERR_DEVICE, M);
    } else {
      // `units` consecutive tiles or row groups; a barrier between them
      // (each pass reuses the block's shared memory from the start)
#pragma unroll 1
      for (int u = 0; u < units; ++u) {
        if (u) __syncthreads();
        if constexpr (MODE == MODE_HERM) {
          if (type == T_A) run_A_herm<M, V>(a, x, y + u, sm, rt);
          else if (type == T_B) run_B_herm<M, V>(a, x, y + u, sm, rt);
          else run_C_herm<M, V>(a, x, y + u, sm, rt);
        } else if constexpr (MODE == MODE_TERN) {
          if (type == T_A) run_A_tern<M, V>(a, x, y + u, sm, rt);
          else if (type == T_B) run_B<M, V, true>(a, x, y + u, sm, rt);
          else run_C<M, V, true>(a, x, y + u, sm, rt);
        } else {
          if (type == T_A) run_A<M, V>(a, x, y + u, sm, rt);
          else if (type == T_B) run_B<M, V, false>(a, x, y + u, sm, rt);
          else run_C<M, V, false>(a, x, y + u, sm, rt);
        }
      }
    }
  }
}

// bounded wait until *c >= need (thread 0 only); false on timeout.  A wait
// that was not satisfied at once adds its cycles to the header's counters.
__device__ __forceinline__ bool wait_geq(const uint32_t* c, uint32_t need, WorkHeader* hdr, long long limit) {
  const long long t0 = clock64();
  for (int it = 0;; ++it) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(c) : "memory");
    const long long dt = clock64() - t0;
    if (v >= need) {
      if (it > 0) {
        atomicAdd(&hdr->waited, 1u);
        atomicAdd(&hdr->wait_cycles, (unsigned long long)dt);
      }
      return true;
    }
    if (dt > limit) return false;
    __nanosleep(256);
  }
}

// byte offset of the root tables of size code `code` in shared memory
__device__ __forceinline__ int roots_off_of(int code, bool herm) {
  if (!herm) return 0;
  switch (code) {
#define DC_FX_OFF(c) \
    case c: return Shape<size_of_code(c)>::herm_behind ? Shape<size_of_code(c)>::herm_off : 0;
    DC_FX_OFF(0) DC_FX_OFF(1) DC_FX_OFF(2) DC_FX_OFF(3) DC_FX_OFF(4) DC_FX_OFF(5) DC_FX_OFF(6) DC_FX_OFF(7)
    DC_FX_OFF(8) DC_FX_OFF(9) DC_FX_OFF(10) DC_FX_OFF(11) DC_FX_OFF(12) DC_FX_OFF(13) DC_FX_OFF(14)
    DC_FX_OFF(15) DC_FX_OFF(16) DC_FX_OFF(17) DC_FX_OFF(18) DC_FX_OFF(19) DC_FX_OFF(20) DC_FX_OFF(21)
    DC_FX_OFF(22) DC_FX_OFF(23) DC_FX_OFF(24) DC_FX_OFF(25) DC_FX_OFF(26) DC_FX_OFF(27) DC_FX_OFF(28)
    DC_FX_OFF(29) DC_FX_OFF(30)
#undef DC_FX_OFF
    default: return 0;
  }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, kBlocksPerSM) fx_kernel(const __grid_constant__ FxArgs a) {
  unsigned char* smem_raw = fx_smem;
  C* rts = (C*)smem_raw;
  C* sm = rts + kRootsMax;
  __shared__ Task s_task;
  __shared__ int s_ok;
  int cur = -1;
  Roots<C> rt{rts, rts, 0, 0};
  // thread 0 takes the next queue index while the current task runs
  uint32_t next = 0;
  if (threadIdx.x == 0) next = atomicAdd(&a.hdr->counter, 1u);
  long long t_end = clock64();   // thread 0: end of the previous task (start of the launch at first)
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const uint32_t idx = next;
      Task t;
      t.kc = -1;
      int ok = 1;
      if (idx < (uint32_t)a.ntasks) {
        t = a.tasks[idx];
        next = atomicAdd(&a.hdr->counter, 1u);
        if (t.widx >= 0 && !wait_geq(a.cnt + t.widx, t.wneed, a.hdr, a.wait_limit)) {
          ok = 0;
          record_error(a.hdr, DC_ERR_TIMEOUT, (int)idx);
        }
      }
      s_task = t;
      s_ok = ok;
    }
    __syncthreads();
    const Task t = s_task;
    if (t.kc < 0 || !s_ok) break;
    const int code = t.kc & 255, type = (t.kc >> 8) & 255, units = max(1, t.kc >> 16);
    const long long t_got = clock64();
    if (code != cur) {
      // lo = zeta_TN^b (b < 2^sh), hi = zeta_TN^(a 2^sh), from the full table
      const int TN = mode_q(MODE) * size_of_code(code % kCodeStride);
      const int sh = roots_sh(TN), nlo = 1 << sh, cnt = roots_count(TN);
      const C* tab = (const C*)a.tab[code];
      // the low table always starts shared memory; the high one follows it,
      // or sits behind the task data for the Hermitian level-2 sizes
      const int hoff = roots_off_of(code % kCodeStride, mode_tables_3m(MODE));
      C* hi = hoff ? (C*)(smem_raw + hoff) : rts + nlo;
      // and the size's stage tables (a contiguous copy) behind its task data
      const C* stab = (const C*)a.stab[code];
      C* sdst = (C*)(smem_raw + a.stab_off[code]);
      // (asynchronous copies: a thread's entries are all in flight at once,
      // one L2 round trip per switch instead of one per entry it copies)
      for (int e = threadIdx.x; e < cnt + a.stab_n[code]; e += kThreads) {
        if (e < cnt) cp_async_elem(e < nlo ? rts + e : hi + (e - nlo), tab + (e < nlo ? e : (e - nlo) << sh));
        else cp_async_elem(sdst + (e - cnt), stab + (e - cnt));
      }
      cp_async_commit();
      cp_async_wait_all();
      rt = Roots<C>{rts, hi, sh, nlo - 1};
      cur = code;
      __syncthreads();
    }
    const long long t_start = clock64();
    if (threadIdx.x == 0) {
      atomicAdd(&a.hdr->handover_cycles, (unsigned long long)(t_got - t_end));
      atomicAdd(&a.hdr->table_cycles, (unsigned long long)(t_start - t_got));
    }
    if (code < kCodeStride) {
      switch (code) {
#define DC_FX_CASE(c) \
        case c: run_size<size_of_code(c), 0, MODE>(&a, type, t.a, t.b, units, sm, rt); break;
        DC_FX_CASE(0) DC_FX_CASE(1) DC_FX_CASE(2) DC_FX_CASE(3) DC_FX_CASE(4) DC_FX_CASE(5)
        DC_FX_CASE(6) DC_FX_CASE(7) DC_FX_CASE(8) DC_FX_CASE(9) DC_FX_CASE(10)
        DC_FX_CASE(11) DC_FX_CASE(12) DC_FX_CASE(13) DC_FX_CASE(14) DC_FX_CASE(15)
        DC_FX_CASE(16) DC_FX_CASE(17) DC_FX_CASE(18) DC_FX_CASE(19) DC_FX_CASE(20)
        DC_FX_CASE(21) DC_FX_CASE(22) DC_FX_CASE(23) DC_FX_CASE(24) DC_FX_CASE(25)
        DC_FX_CASE(26) DC_FX_CASE(27) DC_FX_CASE(28) DC_FX_CASE(29) DC_FX_CASE(30)
#undef DC_FX_CASE
        default: break;
      }
    } else if constexpr (kVariantKind(MODE)) {
      // variant 1 of the two-level sizes (the other split)
      switch (code - kCodeStride) {
#define DC_FX_CASE1(c) \
        case c: run_size<size_of_code(c), 1, MODE>(&a, type, t.a, t.b, units, sm, rt); break;
        DC_FX_CASE1(7) DC_FX_CASE1(8) DC_FX_CASE1(9) DC_FX_CASE1(10) DC_FX_CASE1(18) DC_FX_CASE1(19)
        DC_FX_CASE1(20) DC_FX_CASE1(28) DC_FX_CASE1(29) DC_FX_CASE1(30)
#undef DC_FX_CASE1
        default: break;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      // the barrier above orders every thread's stores of the task before
      // this release at GPU scope
      if (t.sidx >= 0)
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(a.cnt + t.sidx), "r"(units) : "memory");
      // per-type time, for tracing where a launch spends its cycles
      t_end = clock64();
      atomicAdd(&a.hdr->type_cycles[type & 3], (unsigned long long)(t_end - t_start));
      atomicAdd(&a.hdr->type_count[type & 3], 1u);
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// Each kind's kernel is compiled in a translation unit of its own (built with
// DC_FX_MODE set), so the kinds compile in parallel; the planner below is
// built once, without DC_FX_MODE, and reaches the kernels through these.
dc_status prepare_mode0(int smem, int* blocks);
dc_status prepare_mode1(int smem, int* blocks);
dc_status prepare_mode2(int smem, int* blocks);
dc_status prepare_mode3(int smem, int* blocks);
dc_status prepare_mode4(int smem, int* blocks);
dc_status prepare_mode5(int smem, int* blocks);
dc_status launch_mode0(const FxArgs& a, int grid, int smem, cudaStream_t s);
dc_status launch_mode1(const FxArgs& a, int grid, int smem, cudaStream_t s);
dc_status launch_mode2(const FxArgs& a, int grid, int smem, cudaStream_t s);
dc_status launch_mode3(const FxArgs& a, int grid, int smem, cudaStream_t s);
dc_status launch_mode4(const FxArgs& a, int grid, int smem, cudaStream_t s);
dc_status launch_mode5(const FxArgs& a, int grid, int smem, cudaStream_t s);

#if defined(DC_FX_MODE)
#define DC_FX_CAT2(a, b) a##b
#define DC_FX_CAT(a, b) DC_FX_CAT2(a, b)
dc_status DC_FX_CAT(prepare_mode, DC_FX_MODE)(int smem, int* blocks) {
  DC_CUDA_TRY(cudaFuncSetAttribute(fx_kernel<DC_FX_MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  DC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fx_kernel<DC_FX_MODE>, kThreads, smem));
  return DC_OK;
}
dc_status DC_FX_CAT(launch_mode, DC_FX_MODE)(const FxArgs& a, int grid, int smem, cudaStream_t s) {
  fx_kernel<DC_FX_MODE><<<grid, kThreads, smem, s>>>(a);
  DC_CUDA_TRY(cudaGetLastError());
  return DC_OK;
}
#undef DC_FX_CAT
#undef DC_FX_CAT2
#else
namespace {
template <int V, int... Cs> struct CodeTable {
  static void fill(int* lvl, int* per, int* l1, int* l2, int* w, int* na, int* nb, int* nbh, int* smem, int* tabn,
                   int* taboff) {
    int k = V * kCodeStride;
    ((lvl[k] = Shape<size_of_code(Cs), V>::l1 ? 1 : 2, per[k] = Shape<size_of_code(Cs), V>::G,
      l1[k] = Shape<size_of_code(Cs), V>::L1, l2[k] = Shape<size_of_code(Cs), V>::L2,
      w[k] = Shape<size_of_code(Cs), V>::W, na[k] = Shape<size_of_code(Cs), V>::nA,
      nb[k] = Shape<size_of_code(Cs), V>::nB, nbh[k] = Shape<size_of_code(Cs), V>::nBh,
      smem[k] = Shape<size_of_code(Cs), V>::total, tabn[k] = Shape<size_of_code(Cs), V>::tab_entries,
      taboff[k] = Shape<size_of_code(Cs), V>::tab_off, ++k),
     ...);
  }
};
// per kernel code (size code + kCodeStride * variant); variant 1 entries of
// sizes without one repeat variant 0 and are never used
struct Tables {
  int lvl[kNumCodes], per[kNumCodes], l1[kNumCodes], l2[kNumCodes], w[kNumCodes], na[kNumCodes],
      nb[kNumCodes], nbh[kNumCodes], smem[kNumCodes], tabn[kNumCodes], taboff[kNumCodes];
  Tables() {
    std::memset(this, 0, sizeof(*this));
    CodeTable<0, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25,
              26, 27, 28, 29, 30>::fill(lvl, per, l1, l2, w, na, nb, nbh, smem, tabn, taboff);
    CodeTable<1, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25,
              26, 27, 28, 29, 30>::fill(lvl, per, l1, l2, w, na, nb, nbh, smem, tabn, taboff);
  }
};

// the stage tables of a kernel code, one block
template <int M, int V> __global__ void gen_tabs_kernel(C* st) { gen_size_tabs<M, V>(st); }
std::mutex g_tab_mu;
std::map<std::pair<int, int>, void*> g_stage_tabs;   // (device, kernel code) -> tables
const Tables& tables() {
  static Tables t;
  return t;
}
}  // namespace

int size_code(int64_t m) {
  for (int c = 0; c < kNumSizes; ++c)
    if (size_of_code(c) == m) return c;
  return -1;
}
int64_t code_size(int code) { return size_of_code(code % kCodeStride); }
bool code_level1(int code) { return tables().lvl[code] == 1; }
bool code_ok(int code, int mode) {
  if (code < 0 || code >= kNumCodes || code % kCodeStride >= kNumSizes) return false;
  return code < kCodeStride || (kVariantKind(mode) && two_level_code(code - kCodeStride));
}
int code_smem(int code) { return tables().smem[code]; }
void code_tabs(int code, int* entries, int* byte_off) {
  *entries = tables().tabn[code];
  *byte_off = tables().taboff[code];
}

dc_status stage_tables(int code, const void** out) {
  *out = nullptr;
  const int n = tables().tabn[code];
  if (n == 0) return DC_OK;
  int dev = 0;
  DC_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_tab_mu);
  auto it = g_stage_tabs.find({dev, code});
  if (it != g_stage_tabs.end()) {
    *out = it->second;
    return DC_OK;
  }
  void* p = nullptr;
  DC_CUDA_TRY(cudaMalloc(&p, (size_t)n * sizeof(C)));
  cudaStream_t s;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaFree(p);
    dc_set_last_cuda_error(e);
    return DC_ERR_CUDA;
  }
  switch (code) {
#define DC_FX_GEN(c)                                                                   \
    case c: gen_tabs_kernel<size_of_code(c), 0><<<1, kThreads, 0, s>>>((C*)p); break;  \
    case c + kCodeStride: gen_tabs_kernel<size_of_code(c), 1><<<1, kThreads, 0, s>>>((C*)p); break;
    DC_FX_GEN(7) DC_FX_GEN(8) DC_FX_GEN(9) DC_FX_GEN(10) DC_FX_GEN(18) DC_FX_GEN(19) DC_FX_GEN(20)
    DC_FX_GEN(28) DC_FX_GEN(29) DC_FX_GEN(30)
#undef DC_FX_GEN
    default: break;
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (e != cudaSuccess) {
    cudaFree(p);
    dc_set_last_cuda_error(e);
    return DC_ERR_CUDA;
  }
  g_stage_tabs[{dev, code}] = p;
  *out = p;
  return DC_OK;
}
void code_shape(int code, int* level, int* per_task, int* L1, int* L2, int* W) {
  const Tables& t = tables();
  *level = t.lvl[code];
  *per_task = t.lvl[code] == 1 ? t.per[code] : 1;
  *L1 = t.lvl[code] == 1 ? 0 : t.l1[code];
  *L2 = t.lvl[code] == 1 ? 0 : t.l2[code];
  *W = t.lvl[code] == 1 ? 0 : t.w[code];
}

bool build_plan(const int64_t* m, int32_t n, const int64_t* off, const Schedule& sc, int mode, HostPlan* out) {
  const int batch_target = std::max(1, sc.batch_target);
  const Tables& tb = tables();
  HostPlan& P = *out;
  P = HostPlan{};
  std::map<int, std::vector<int32_t>> l1_by_code;
  std::vector<std::pair<int, int32_t>> big;   // (code, instance)
  std::vector<bool> used(kNumCodes, false);
  P.l1tmp.assign((size_t)n, 0);
  for (int32_t i = 0; i < n; ++i) {
    int c = size_code(m[i]);
    if (c < 0) return false;
    if ((mode == MODE_TERN && tb.lvl[c] == 1) ||
        ((mode == MODE_PAIR || mode == MODE_HDOT2 || mode == MODE_TERN4) && tb.lvl[c] == 2))
      return false;
    // the kernel code: variant 1 of the split where the schedule asks for it
    if (((sc.variants >> c) & 1u) && code_ok(c + kCodeStride, mode)) c += kCodeStride;
    used[c] = true;
    if (tb.lvl[c] == 1) {
      l1_by_code[c].push_back(i);
      // in-place partial outputs: one slot per output
      P.l1tmp[i] = (int64_t)P.l1_elems;
      P.l1_elems += (size_t)m[i] * (mode == MODE_PAIR ? 2 : 1);
    } else {
      big.push_back({c, i});
    }
  }
  for (int c = 0; c < kNumCodes; ++c)
    if (used[c]) {
      P.codes.push_back(c);
      P.smem = std::max(P.smem, code_smem(c));
    }

  // level-1 tasks, largest estimated cost first
  struct L1T { double cost; int code; std::vector<int32_t> ids; };
  std::vector<L1T> l1t;
  for (auto& kv : l1_by_code) {
    const int c = kv.first, per = tb.per[c];
    const double ms = (double)size_of_code(c % kCodeStride);
    for (size_t s = 0; s < kv.second.size(); s += per) {
      L1T t;
      t.code = c;
      t.ids.assign(kv.second.begin() + s, kv.second.begin() + std::min(kv.second.size(), s + per));
      t.cost = (double)t.ids.size() * ms * (std::log2(ms) + 4.0);
      l1t.push_back(std::move(t));
    }
  }
  // largest sizes first and each size's tasks together: blocks that run at
  // the same time then run the same code (one size's code is tens of KB of
  // straight-line instructions) and refill their root tables less often
  std::stable_sort(l1t.begin(), l1t.end(), [](const L1T& x, const L1T& y) {
    const int mx = size_of_code(x.code % kCodeStride), my = size_of_code(y.code % kCodeStride);
    return mx != my ? mx > my : x.cost > y.cost;
  });
  std::vector<Task> l1tasks;
  for (auto& t : l1t) {
    Task k{(T_L1 << 8) | t.code, (int32_t)P.order.size(), (int32_t)t.ids.size(), -1, 0, -1};
    P.order.insert(P.order.end(), t.ids.begin(), t.ids.end());
    l1tasks.push_back(k);
  }

  // level-2 instances, largest first, in batches of about batch_target column tiles
  std::stable_sort(big.begin(), big.end(), [](const std::pair<int, int32_t>& x, const std::pair<int, int32_t>& y) {
    return size_of_code(x.first % kCodeStride) > size_of_code(y.first % kCodeStride);
  });
  const int n2 = (int)big.size();
  std::vector<std::vector<int>> batches;
  std::vector<int64_t> batch_elems;
  {
    int tiles = 0;
    for (int l = 0; l < n2; ++l) {
      if (batches.empty() || tiles >= std::max(1, batch_target)) {
        batches.emplace_back();
        batch_elems.push_back(0);
        tiles = 0;
      }
      batches.back().push_back(l);
      tiles += tb.na[big[l].first];
    }
  }
  const int nbat = (int)batches.size();
  int64_t region = 0;
  for (int k = 0; k < nbat; ++k) {
    int64_t s = 0;
    for (int l : batches[k]) s += 4 * (int64_t)size_of_code(big[l].first % kCodeStride);
    region = std::max(region, s);
  }
  P.l2.resize(n2);
  std::vector<uint32_t> batch_c(nbat, 0);
  for (int k = 0; k < nbat; ++k) {
    int64_t o = (int64_t)(k % 4) * region;
    for (int l : batches[k]) {
      const int c = big[l].first;
      P.l2[l].off = off[big[l].second];
      P.l2[l].scr = o;
      o += 4 * (int64_t)size_of_code(c % kCodeStride);
      batch_c[k] += (uint32_t)tb.na[c];
    }
  }
  P.scratch = (size_t)(nbat ? std::min(nbat, 4) : 0) * (size_t)region;
  P.ncnt = (size_t)2 * n2 + nbat;
  auto emit = [&](int type, int k) {
    for (int l : batches[k]) {
      const int c = big[l].first;
      const int nbc = mode == MODE_HERM ? tb.nbh[c] : tb.nb[c];
      const int cnt = type == T_B ? nbc : tb.na[c];
      const int grp = std::max(1, std::min(sc.units, kMaxUnits));
      for (int u = 0; u < cnt; u += grp) {
        const int n = std::min(grp, cnt - u);
        Task t{(n << 16) | (type << 8) | c, l, u, -1, 0, -1};
        if (type == T_A) {
          if (k >= 4) { t.widx = 2 * n2 + (k - 4); t.wneed = batch_c[k - 4]; }
          t.sidx = 2 * l;
        } else if (type == T_B) {
          t.widx = 2 * l; t.wneed = (uint32_t)tb.na[c]; t.sidx = 2 * l + 1;
        } else {
          t.widx = 2 * l + 1; t.wneed = (uint32_t)nbc; t.sidx = 2 * n2 + k;
        }
        P.tasks.push_back(t);
      }
    }
  };
  size_t li = 0;
  auto take_l1 = [&](size_t k) {
    for (size_t e = 0; e < k && li < l1tasks.size(); ++e) P.tasks.push_back(l1tasks[li++]);
  };
  if (sc.l1_mode == 2) take_l1(l1tasks.size());
  // mode 1: the larger half of the level-1 tasks, spread evenly over the
  // pipeline, fills the waits between dependent passes
  const size_t spread = sc.l1_mode == 1 ? l1tasks.size() / 2 : 0;
  for (int s = 0; s < nbat; ++s) {
    emit(T_A, s);
    if (s >= 1) emit(T_B, s - 1);
    if (s >= 2) emit(T_C, s - 2);
    if (spread) take_l1(spread * (size_t)(s + 1) / (size_t)nbat - li);
  }
  // drain the pipeline with level-1 work between the last passes
  const size_t chunk = (size_t)batch_target * 2;
  if (nbat >= 1) {
    take_l1(chunk);
    emit(T_B, nbat - 1);
    if (nbat >= 2) emit(T_C, nbat - 2);
    take_l1(chunk);
    emit(T_C, nbat - 1);
  }
  take_l1(l1tasks.size());
  return true;
}

dc_status prepare_kernel(int smem, int* blocks_per_sm) {
  int bmin = 1 << 20;
  for (auto prep : {prepare_mode0, prepare_mode1, prepare_mode2, prepare_mode3, prepare_mode4, prepare_mode5}) {
    int b = 0;
    const dc_status st = prep(smem, &b);
    if (st != DC_OK) return st;
    bmin = std::min(bmin, b);
  }
  if (bmin < 1) return DC_ERR_SIZE;
  *blocks_per_sm = bmin;
  return DC_OK;
}

dc_status launch(const FxArgs& a, int grid, int smem, cudaStream_t s) {
  switch (a.mode) {
    case MODE_COMPLEX: return launch_mode0(a, grid, smem, s);
    case MODE_HERM: return launch_mode1(a, grid, smem, s);
    case MODE_TERN: return launch_mode2(a, grid, smem, s);
    case MODE_PAIR: return launch_mode3(a, grid, smem, s);
    case MODE_HDOT2: return launch_mode4(a, grid, smem, s);
    case MODE_TERN4: return launch_mode5(a, grid, smem, s);
    default: return DC_ERR_ARG;
  }
}
#endif  // DC_FX_MODE

}  // namespace DC_FX_P
}  // namespace fx
}  // namespace dc

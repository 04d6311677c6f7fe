// Host-side planning for the 1D kernels (see plan.h).
#include <algorithm>
#include <cmath>

#include "plan.h"

namespace dc {

KindShape kind_shape(int kind) {
  switch (kind) {
    case K_COMPLEX:       return {2, 2, 1, 2, 1};
    case K_HERMITIAN:     return {3, 1, 1, 2, 1};
    case K_TERNARY:       return {2, 2, 1, 3, 1};
    case K_COMPLEX_ADJ:   return {2, 3, 2, 3, 2};
    case K_HERMITIAN_ADJ: return {3, 2, 2, 3, 2};
    case K_HERMITIAN_PAIR: return {3, 2, 2, 3, 2};
    case K_COMPLEX_DOT2:  return {2, 4, 1, 4, 1};
    case K_HERMITIAN_DOT2: return {3, 2, 1, 4, 1};
  }
  return {0, 0, 0, 0, 0};
}

// Ternary sub-transforms are real transforms of size 2m done as complex
// transforms of length L = 2m with roots zeta_{4m} (Sec. 4.2).
int64_t kind_L(int kind, int64_t m) { return kind == K_TERNARY ? 2 * m : m; }
int64_t kind_TN(int kind, int64_t m) {
  switch (kind) {
    case K_HERMITIAN:
    case K_HERMITIAN_ADJ:
    case K_HERMITIAN_PAIR:
    case K_HERMITIAN_DOT2: return 3 * m;
    case K_TERNARY:       return 4 * m;
    default:              return 2 * m;
  }
}

// L = 2^a 3^b 5^c (any a, b, c >= 0)
static bool factor(int64_t L, int* a, int* b, int* c) {
  if (L < 1) return false;
  *a = *b = *c = 0;
  while (L % 2 == 0) { L /= 2; ++*a; }
  while (L % 3 == 0) { L /= 3; ++*b; }
  while (L % 5 == 0) { L /= 5; ++*c; }
  return L == 1;
}

static int lcm(int x, int y) {
  int a = x, b = y;
  while (b) { int t = a % b; a = b; b = t; }
  return x / a * y;
}

static bool e_supported(int E) {
  static const int ok[] = {1, 2, 3, 4, 5, 6, 8, 10, 12, 15, 16, 20, 24, 30};
  for (int v : ok) if (v == E) return true;
  return false;
}

bool make_fft_plan(int L, int emax, FftPlan* out) {
  int a, b, c;
  if (!factor(L, &a, &b, &c)) return false;
  static const int pmax_opts[] = {16, 8, 4, 2};
  for (int pmax : pmax_opts) {
    if (pmax > emax) continue;
    FftPlan p{};
    p.L = L;
    int lg = 0;
    while ((1 << (lg + 1)) <= pmax) ++lg;          // log2(pmax)
    if (b + c + a / lg + 1 > kMaxStages) continue;
    int ns = 0;
    for (int i = 0; i < c; ++i) p.r[ns++] = 5;
    for (int i = 0; i < b; ++i) p.r[ns++] = 3;
    int rem = a;
    while (rem >= lg) { p.r[ns++] = (int8_t)(1 << lg); rem -= lg; }
    if (rem > 0) p.r[ns++] = (int8_t)(1 << rem);
    int E = 1;
    for (int s = 0; s < ns; ++s) E = lcm(E, p.r[s]);
    if (!e_supported(E) || E > emax) continue;
    p.ns = ns;
    p.E = E;
    p.tpt = L / E;
    *out = p;
    return true;
  }
  return false;
}

int64_t fft_flops(int L) {
  return L > 1 ? (int64_t)std::llround(5.0 * L * std::log2((double)L)) : 0;
}

static int largest_divisor_at_most(int n, int cap) {
  for (int d = std::min(n, cap); d >= 1; --d) if (n % d == 0) return d;
  return 1;
}

// Plan of the fused engine (fft2.cuh): one E per size family (FP32: 16 for
// 2^a, 12 for 2^a 3^b, 20 for 2^a 5^c; FP64: 8, 12, 10; larger E spills
// registers), the powers of two first and the odd radices (3 or 5, repeated
// b or c times) last.  Returns a plan with E = 0 (DFT by definition, one
// thread per element) when L is not a multiple of E, and when both 3 and 5
// divide L (no E of the engine holds both radices).
bool make_fused_plan(int L, int dsize, FftPlan* out) {
  int a, b, c;
  if (!factor(L, &a, &b, &c)) return false;
  FftPlan p{};
  p.L = L;
  int E, pmax;
  if (dsize == 8) {
    if (c) { E = 20; pmax = 4; } else if (b) { E = 12; pmax = 4; } else { E = 16; pmax = 16; }
  } else {
    if (c) { E = 10; pmax = 2; } else if (b) { E = 12; pmax = 4; } else { E = 8; pmax = 8; }
  }
  if (L % E != 0 || L < E || (b && c)) {
    p.E = 0;
    p.tpt = L;
    p.ns = 0;
    *out = p;
    return true;
  }
  // powers of two first, the odd radices last (the forward transform uses
  // the same order); stages after the first odd one start at strides Ns
  // that are not powers of two
  int lg = 0;
  while ((1 << (lg + 1)) <= pmax) ++lg;
  int rs[64];
  int ns = 0;
  int rem = a;
  while (rem >= lg) { rs[ns++] = 1 << lg; rem -= lg; }
  if (rem > 0) rs[ns++] = 1 << rem;
  for (int i = 0; i < b; ++i) rs[ns++] = 3;
  for (int i = 0; i < c; ++i) rs[ns++] = 5;
  if (ns > kMaxStages) return false;
  for (int s = 0; s < ns; ++s) p.r[s] = (int8_t)rs[s];
  if (ns == 1) {          // one stage: the DFT by definition is as cheap
    p.E = 0;
    p.tpt = L;
    p.ns = 0;
    *out = p;
    return true;
  }
  p.ns = ns;
  p.E = E;
  p.tpt = L / E;
  *out = p;
  return true;
}

static int64_t padded(int64_t n, int dsize) { return n + (n >> (dsize == 8 ? 4 : 3)) + 1; }

// bytes of the two shared-memory root tables for TN (rounded to an even
// number of entries), as the kernel lays them out
static int64_t roots_bytes(int64_t TN, int dsize) {
  int lg = 0;
  while ((1ll << lg) < TN) ++lg;
  const int sh = (lg + 1) / 2;
  const int64_t S = 1ll << sh;
  const int64_t ent = S + ((TN + S - 1) >> sh) + 2;
  return ((ent + 1) & ~1ll) * dsize;
}

bool make_cfg(int kind, int64_t m, int dsize, int threads, int smem_max, int force_level,
              CfgDev* out) {
  const KindShape ks = kind_shape(kind);
  if (ks.q == 0 || m < 1) return false;
  const int64_t L = kind_L(kind, m), TN = kind_TN(kind, m);
  if (L > (1 << 20)) return false;
  int a, b, c;
  if (!factor(L, &a, &b, &c)) return false;
  CfgDev cfg{};
  cfg.m = (int32_t)m;
  cfg.L = (int32_t)L;
  cfg.TN = (int32_t)TN;
  const int64_t rb = roots_bytes(TN, dsize);
  const int64_t avail = smem_max - rb;

  if (force_level != 2) {
    FftPlan p;
    if (make_fused_plan((int)L, dsize, &p) && p.tpt <= threads) {
      const int64_t per = p.E ? (ks.narr * padded(L, dsize) + ks.nfwd * padded(m, dsize)) * dsize
                              : (ks.narr * L + ks.nfwd * m) * dsize;
      const int64_t nt = std::min<int64_t>(threads / p.tpt, avail / per);
      if (nt >= 1) {
        cfg.level = 1;
        cfg.p = p;
        cfg.nt = (int32_t)nt;
        cfg.smem = (int32_t)(rb + nt * per);
        *out = cfg;
        return true;
      }
    }
    if (force_level == 1) return false;
  }
  // two-level: L = L1 * L2 with L2 <= L1, both with fused (non-direct) plans
  int bestL2 = 0;
  FftPlan pr{}, pc{};
  for (int64_t L2 = 2; L2 * L2 <= L; ++L2) {
    if (L % L2) continue;
    FftPlan tr, tc;
    if (!make_fused_plan((int)(L / L2), dsize, &tr) || !make_fused_plan((int)L2, dsize, &tc)) continue;
    if (!tr.E || !tc.E || tr.tpt > threads || tc.tpt > threads) continue;
    bestL2 = (int)L2;
    pr = tr;
    pc = tc;
  }
  if (bestL2 < 1) return false;
  const int L2 = bestL2, L1 = (int)(L / L2);
  const int64_t colbytes = (int64_t)L2 * dsize;
  const int64_t rowbytes = padded(L1, dsize) * dsize;
  const int wcap = (int)std::min<int64_t>(threads / pc.tpt, avail / ((1 + ks.nfwd) * colbytes));
  const int ncap = (int)std::min<int64_t>(threads / pr.tpt, avail / (ks.narr * rowbytes));
  if (wcap < 1 || ncap < 1) return false;
  const int w = largest_divisor_at_most(L1, std::min(wcap, 64));
  const int nr = largest_divisor_at_most(L2, ncap);
  cfg.level = 2;
  cfg.L1 = L1;
  cfg.L2 = L2;
  cfg.w = w;
  cfg.nr = nr;
  cfg.pr = pr;
  cfg.pc = pc;
  cfg.nt = 1;
  cfg.smem = (int32_t)(rb + std::max<int64_t>((1 + ks.nfwd) * w * colbytes, ks.narr * nr * rowbytes));
  *out = cfg;
  return true;
}

int enumerate_cfgs(int kind, int64_t m, int dsize, int threads, int smem_max, CfgDev* out, int maxn) {
  const KindShape ks = kind_shape(kind);
  int n = 0;
  CfgDev base;
  if (!make_cfg(kind, m, dsize, threads, smem_max, 0, &base)) return 0;
  out[n++] = base;
  const int64_t L = kind_L(kind, m), TN = kind_TN(kind, m);
  const int64_t rb = roots_bytes(TN, dsize), avail = smem_max - rb;
  // level 1 with fewer instances per block (more blocks per SM)
  if (base.level == 1) {
    for (int nt = base.nt / 2; nt >= 1 && n < maxn; nt /= 2) {
      CfgDev c = base;
      const int64_t per = (base.smem - rb) / base.nt;
      c.nt = nt;
      c.smem = (int32_t)(rb + nt * per);
      out[n++] = c;
    }
  }
  // level 2 with other splits and tile widths (also for sizes that fit level 1)
  for (int64_t L2 = 2; L2 * L2 <= L && n < maxn; ++L2) {
    if (L % L2) continue;
    FftPlan pr, pc;
    if (!make_fused_plan((int)(L / L2), dsize, &pr) || !make_fused_plan((int)L2, dsize, &pc)) continue;
    if (!pr.E || !pc.E || pr.tpt > threads || pc.tpt > threads) continue;
    const int L1 = (int)(L / L2);
    const int64_t colbytes = L2 * dsize, rowbytes = padded(L1, dsize) * dsize;
    const int wcap = (int)std::min<int64_t>(threads / pc.tpt, avail / ((1 + ks.nfwd) * colbytes));
    const int ncap = (int)std::min<int64_t>(threads / pr.tpt, avail / (ks.narr * rowbytes));
    if (wcap < 1 || ncap < 1) continue;
    const int nr = largest_divisor_at_most((int)L2, ncap);
    for (int wmax : {64, 32, 16, 8}) {
      if (n >= maxn) break;
      const int w = largest_divisor_at_most(L1, std::min(wcap, wmax));
      bool dup = false;
      for (int q = 0; q < n; ++q)
        if (out[q].level == 2 && out[q].L2 == L2 && out[q].w == w) dup = true;
      if (dup) continue;
      CfgDev c{};
      c.level = 2; c.m = (int32_t)m; c.L = (int32_t)L; c.TN = (int32_t)TN;
      c.L1 = L1; c.L2 = (int32_t)L2; c.w = w; c.nr = nr; c.pr = pr; c.pc = pc; c.nt = 1;
      c.smem = (int32_t)(rb + std::max<int64_t>((1 + ks.nfwd) * w * colbytes, ks.narr * nr * rowbytes));
      out[n++] = c;
    }
  }
  return n;
}

size_t cfg_scratch_bytes(int kind, const CfgDev& c, int dsize) {
  if (c.level != 2) return 0;
  const KindShape ks = kind_shape(kind);
  return (size_t)ks.q * ks.narr * (size_t)c.L * dsize;
}

}  // namespace dc

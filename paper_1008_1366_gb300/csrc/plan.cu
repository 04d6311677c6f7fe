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
    case K_HERMITIAN_PAIR: return 3 * m;
    case K_TERNARY:       return 4 * m;
    default:              return 2 * m;
  }
}

static bool factor(int64_t L, int* a, int* b, int* c) {
  if (L < 1) return false;
  *a = *b = *c = 0;
  while (L % 2 == 0) { L /= 2; ++*a; }
  while (L % 3 == 0) { L /= 3; ++*b; }
  while (L % 5 == 0) { L /= 5; ++*c; }
  return L == 1 && *b <= 1 && *c <= 1;
}

static int lcm(int x, int y) {
  int a = x, b = y;
  while (b) { int t = a % b; a = b; b = t; }
  return x / a * y;
}

static bool e_supported(int E) {
  static const int ok[] = {1, 2, 3, 4, 5, 6, 8, 10, 12, 16, 20, 24};
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
    int ns = 0;
    for (int i = 0; i < c; ++i) p.r[ns++] = 5;
    for (int i = 0; i < b; ++i) p.r[ns++] = 3;
    int lg = 0;
    while ((1 << (lg + 1)) <= pmax) ++lg;          // log2(pmax)
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

bool make_cfg(int kind, int64_t m, int dsize, int threads, int smem_max, int force_level,
              CfgDev* out) {
  const KindShape ks = kind_shape(kind);
  if (ks.q == 0 || m < 1) return false;
  const int64_t L = kind_L(kind, m), TN = kind_TN(kind, m);
  if (L > (1 << 20)) return false;
  int a, b, c;
  if (!factor(L, &a, &b, &c)) return false;
  const int emax = dsize == 8 ? 24 : 12;   // FP64: radix <= 8, E <= 12 (register budget)
  CfgDev cfg{};
  cfg.m = (int32_t)m;
  cfg.L = (int32_t)L;
  cfg.TN = (int32_t)TN;
  const int64_t mout = m;

  if (force_level != 2) {
    FftPlan p;
    if (make_fft_plan((int)L, emax, &p) && p.tpt <= threads) {
      const int64_t per = (int64_t)(ks.narr * L + ks.nfwd * mout) * dsize;
      int64_t nt = std::min<int64_t>(threads / p.tpt, smem_max / per);
      if (nt >= 1) {
        cfg.level = 1;
        cfg.p = p;
        cfg.nt = (int32_t)nt;
        cfg.smem = (int32_t)(nt * per);
        *out = cfg;
        return true;
      }
    }
    if (force_level == 1) return false;
  }
  // two-level: L = L1 * L2 with L2 <= L1, both of the allowed form
  int bestL2 = 0;
  for (int64_t L2 = 1; L2 * L2 <= L; ++L2) {
    if (L % L2) continue;
    int x, y, z;
    if (factor(L2, &x, &y, &z) && factor(L / L2, &x, &y, &z)) bestL2 = (int)L2;
  }
  if (bestL2 < 1) return false;
  const int L2 = bestL2, L1 = (int)(L / L2);
  FftPlan pr, pc;
  if (!make_fft_plan(L1, emax, &pr) || !make_fft_plan(L2, emax, &pc)) return false;
  if (pr.tpt > threads || pc.tpt > threads) return false;
  const int64_t colbytes = (int64_t)L2 * dsize;
  int wcap = (int)std::min<int64_t>(threads / pc.tpt, smem_max / ((1 + ks.nfwd) * colbytes));
  int ncap = (int)std::min<int64_t>(threads / pr.tpt, smem_max / ((int64_t)ks.narr * L1 * dsize));
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
  cfg.smem = (int32_t)std::max<int64_t>((1 + ks.nfwd) * w * colbytes,
                                        (int64_t)ks.narr * nr * L1 * dsize);
  *out = cfg;
  return true;
}

size_t cfg_scratch_bytes(int kind, const CfgDev& c, int dsize) {
  if (c.level != 2) return 0;
  const KindShape ks = kind_shape(kind);
  return (size_t)ks.q * ks.narr * (size_t)c.L * dsize;
}

}  // namespace dc

// Partition of a batch of independent 1D convolutions across ranks (one
// process per GPU) by the longest-processing-time rule: instances in order
// of decreasing cost, each given to the rank with the least load so far.
// The cost of an instance of size m is m log2 m, the operation count of its
// sub-transforms (6 K m log m for the complex case, Sec. 2.1); the rule is
// a scheduling choice with no counterpart in the paper.  Host code only.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "../../include/dealias.h"

namespace {

double cost_of(int64_t m) {
  const double x = (double)m;
  return x * std::max(1.0, std::log2(x));
}

}  // namespace

extern "C" {

dc_status dc_partition_lpt(const int64_t* m, int32_t n, int32_t nranks, int32_t* owner, double* load) {
  if (n < 0 || nranks < 1 || (n > 0 && (!m || !owner))) return DC_ERR_ARG;
  for (int32_t i = 0; i < n; ++i)
    if (m[i] < 1) return DC_ERR_ARG;
  std::vector<int32_t> idx((size_t)n);
  std::iota(idx.begin(), idx.end(), 0);
  // decreasing cost; equal costs in instance order, so the result is a
  // function of the sizes alone
  std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) { return cost_of(m[a]) > cost_of(m[b]); });
  std::vector<double> ld((size_t)nranks, 0.0);
  for (int32_t i : idx) {
    int32_t best = 0;
    for (int32_t r = 1; r < nranks; ++r)
      if (ld[r] < ld[best]) best = r;   // ties: the lowest rank
    owner[i] = best;
    ld[best] += cost_of(m[i]);
  }
  if (load)
    for (int32_t r = 0; r < nranks; ++r) load[r] = ld[r];
  return DC_OK;
}

}  // extern "C"

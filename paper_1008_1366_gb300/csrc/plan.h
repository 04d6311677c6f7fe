// Host-side planning: radix plans for the m-point sub-transforms, tiling of
// the one- and two-level kernels, and the per-size configuration records the
// kernels read.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "fft.cuh"

namespace dc {

enum Kind : int32_t {
  K_COMPLEX = 0,       // binary complex convolution, q = 2 (Sec. 2.1)
  K_HERMITIAN = 1,     // centered Hermitian convolution, q = 3 (Sec. 2.3)
  K_TERNARY = 2,       // centered Hermitian ternary convolution, N = 4m (Sec. 4.2)
  K_COMPLEX_ADJ = 3,   // gradient of K_COMPLEX: correlations with conj partners
  K_HERMITIAN_ADJ = 4, // gradient of K_HERMITIAN
  K_HERMITIAN_PAIR = 5,// two Hermitian convolutions (W, g) and (W, f) sharing W (rows of
                       // the multi-D Hermitian gradient)
  K_COMPLEX_DOT2 = 6,  // f1 * g1 + f2 * g2, complex (Sec. 3, 2D pseudospectral application)
  K_HERMITIAN_DOT2 = 7,// f1 * g1 + f2 * g2, centered Hermitian (same passage)
};
constexpr int kNumKinds = 8;

// Shape of one kind: q residues, NARR shared-memory arrays per residue
// (backward transforms), NFWD forward transforms, NIN inputs, NOUT outputs.
struct KindShape { int q, narr, nfwd, nin, nout; };
KindShape kind_shape(int kind);
// sub-transform length L and root-table length TN for unpadded size m
int64_t kind_L(int kind, int64_t m);
int64_t kind_TN(int kind, int64_t m);

// Per-size configuration read by the 1D kernels (device copy in a plan).
struct CfgDev {
  int32_t level;     // 1: whole transform in shared memory; 2: two-level
  int32_t m;         // unpadded size
  int32_t L, TN;     // sub-transform length and root-table length
  int32_t nt;        // level 1: instances per block
  int32_t L1, L2;    // level 2: L = L1 * L2 (rows of length L1, columns of length L2)
  int32_t w, nr;     // level 2: column-tile width, rows per row tile
  int32_t smem;      // dynamic shared memory bytes this configuration uses
  int32_t pad0;
  const void* tw;    // root table zeta_TN^i (device)
  FftPlan p;         // level 1: length-L plan
  FftPlan pr, pc;    // level 2: row (L1) and column (L2) plans
};

struct Item { int32_t cfg, first, count, pad; };

bool make_fft_plan(int L, int emax, FftPlan* out);     // generic plan (axis passes)
bool make_fused_plan(int L, int dsize, FftPlan* out);  // fused 1D engine
int64_t fft_flops(int L);   // nominal 5 L log2 L

// Chooses a configuration for size m of a kind; returns false when m is not
// of the form 2^a 3^b 5^c with b, c <= 1 (or exceeds the supported range).
// When force_level is 1 or 2 it forces that path (fails if impossible).
bool make_cfg(int kind, int64_t m, int dsize, int threads, int smem_max, int force_level,
              CfgDev* out);

// Candidate configurations for the autotuner: the default first, then
// level 1 with fewer instances per block and level 2 with other splits and
// tile widths.  Returns the number written (<= maxn).
int enumerate_cfgs(int kind, int64_t m, int dsize, int threads, int smem_max, CfgDev* out, int maxn);

// Scratch bytes one block needs for a level-2 configuration.
size_t cfg_scratch_bytes(int kind, const CfgDev& c, int dsize);

}  // namespace dc

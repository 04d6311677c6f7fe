// Host interface of the fixed-shape engine (fixed.cuh, fixed_batched.cu;
// FP32 and FP64 builds): task records, kernel arguments, planning, launch.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace dc {
namespace fx {

constexpr int kNumSizes = 31;   // {2^a, 3*2^a, 5*2^a} in [64, 65536]
// A kernel code names a size and a variant of its two-level split:
// code = size code + kCodeStride * variant (variant 1: FP32 binary complex
// plans, two-level sizes only).
constexpr int kCodeStride = 32;
constexpr int kNumCodes = 2 * kCodeStride;

// task types of the persistent queue
enum : int32_t { T_L1 = 0, T_A = 1, T_B = 2, T_C = 3 };

// kind of convolution a plan runs (one kernel instantiation each)
//   MODE_COMPLEX  binary complex (N = 2m), both levels
//   MODE_HERM     centered Hermitian (N = 3m), both levels, tables of zeta_{3m}
//   MODE_TERN     centered Hermitian ternary of length m = M / 2 on the
//                 M-point sub-transforms (N = 4m), two-level M only
//   MODE_PAIR     rows of a centered Hermitian gradient: inputs (W, f, g) in
//                 (f, g, e), outputs conv(W, g) in h and conv(W, f) in h2,
//                 tables of zeta_{3m}, one-level sizes only
//   MODE_HDOT2    dot product of two centered Hermitian pairs (arrays of
//                 vectors, Sec. 3): inputs (f1, g1, f2, g2) in (f, g, e, e2),
//                 output f1 * g1 + f2 * g2 in h, tables of zeta_{3m},
//                 one-level sizes only
//   MODE_TERN4    centered Hermitian ternary of length m (N = 4m) as four
//                 m-point residues, inputs (f, g, e), output h, tables of
//                 zeta_{4m}, one-level sizes only
enum : int32_t { MODE_COMPLEX = 0, MODE_HERM = 1, MODE_TERN = 2, MODE_PAIR = 3, MODE_HDOT2 = 4, MODE_TERN4 = 5 };
__host__ __device__ constexpr bool mode_tables_3m(int mode) {
  return mode == MODE_HERM || mode == MODE_PAIR || mode == MODE_HDOT2;
}
// the root table of a kind is zeta_{qm}, q = mode_q(kind)
__host__ __device__ constexpr int mode_q(int mode) { return mode_tables_3m(mode) ? 3 : (mode == MODE_TERN4 ? 4 : 2); }

// One queue entry.  kc = units << 16 | type << 8 | size code.  T_L1: a =
// first slot of the order array, b = instance count.  T_A/T_B/T_C: a =
// level-2 instance, b = the first of `units` consecutive column tiles (A, C)
// or row groups (B) the task runs.  Before it starts the task waits until
// cnt[widx] >= wneed (widx < 0: no wait); when done it adds its units (one
// for T_L1) to cnt[sidx] (sidx < 0: none), so thresholds count tiles and row
// groups whatever the grouping.  Every wait names a counter that only tasks
// earlier in the queue advance.
struct Task {
  int32_t kc, a, b, widx;
  uint32_t wneed;
  int32_t sidx;
};

struct L2Inst {
  int64_t off;   // element offset of the instance in f, g, h
  int64_t scr;   // element offset of its four m-element scratch arrays
};

// data pointers are float2 (FP32 engine) or double2 (FP64 engine)
struct FxArgs {
  const void* f;
  const void* g;
  void* h;
  const void* e;           // third input (ternary: e; gradient pair: g; dot product: f2)
  const void* e2;          // fourth input (dot product: g2)
  void* h2;                // second output (gradient pair)
  const int64_t* off;      // per-instance element offsets
  const int32_t* order;    // instance ids of the level-1 tasks
  const Task* tasks;
  int32_t ntasks;
  int32_t pad;
  const L2Inst* l2;
  uint32_t* cnt;           // dependency counters, zero before each launch
  WorkHeader* hdr;         // status word and queue counter, zero before each launch
  void* scratch;
  void* tmp;               // level-1 partial outputs (residue 0) of in-place calls,
  const int64_t* l1tmp;    // tmp + l1tmp[instance]; others keep them in h
  int32_t in_place;        // an output is an input
  int32_t mode;            // MODE_*
  long long wait_limit;    // SM cycles a dependency wait may take before DC_ERR_TIMEOUT
  const void* tab[kNumCodes];     // root tables zeta_{2m}^i, i < 2m, per kernel code
  // stage-twiddle tables per kernel code (null for sizes without): stab_n
  // entries, copied to byte stab_off of the block's shared memory
  const void* stab[kNumCodes];
  int32_t stab_n[kNumCodes];
  int32_t stab_off[kNumCodes];
};

struct HostPlan {
  std::vector<Task> tasks;
  std::vector<L2Inst> l2;
  std::vector<int32_t> order;
  size_t ncnt = 0;          // dependency counters
  size_t scratch = 0;       // scratch elements
  std::vector<int64_t> l1tmp;   // per instance: element offset of its level-1 partial output
  size_t l1_elems = 0;          // elements of the partial-output region
  int smem = 0;             // dynamic shared memory of the launch
  std::vector<int> codes;   // distinct size codes of the plan
};

// Order of the task queue.  batch_target: column tiles per batch of level-2
// instances (the pipeline distance between passes).  l1_mode: where the
// level-1 tasks go (largest first in every mode): 0 after the level-2
// pipeline, 1 the larger half spread over the pipeline and the rest after
// it, 2 before it.  units: column tiles or row groups per pass task (1, 2
// or 4): fewer, longer tasks spend less of the launch handing over.
// variants: bit c set runs the two-level size of size code c in variant 1
// of its split (honoured for FP32 binary complex plans).
struct Schedule {
  int batch_target;
  int l1_mode;
  int units = 1;
  uint32_t variants = 0;
};
constexpr int kMaxUnits = 4;
constexpr int kL1Modes = 3;
constexpr long long kWaitLimit = 1ll << 32;   // about two seconds at 2 GHz

// The interface of one precision of the engine (namespaces f32 and f64).
#define DC_FX_DECLARE                                                                       \
  /* size code of m, or -1 when m is not in the set */                                      \
  int size_code(int64_t m);                                                                 \
  /* whether kernel code `code` (size code + kCodeStride * variant) exists for a kind */    \
  bool code_ok(int code, int mode);                                                         \
  int64_t code_size(int code);                                                              \
  /* instances per task (level 1) or the level-2 split of a size code */                    \
  void code_shape(int code, int* level, int* per_task, int* L1, int* L2, int* W);           \
  /* dynamic shared memory the kernel needs for a size code */                              \
  int code_smem(int code);                                                                  \
  /* stage-twiddle tables of a size code: entries and their shared-memory byte offset */    \
  void code_tabs(int code, int* entries, int* byte_off);                                    \
  /* the stage-twiddle tables of a size code in device memory (generated once per */      \
  /* device in FP64, rounded); null when the size has none */                              \
  dc_status stage_tables(int code, const void** out);                                       \
  /* the task queue for n instances of sizes m[i] at element offsets off[i] for a */      \
  /* convolution kind (MODE_*: row tasks and partial-output slots per instance) */         \
  bool build_plan(const int64_t* m, int32_t n, const int64_t* off, const Schedule& sc,     \
                  int mode, HostPlan* out);                                                 \
  /* kernel attributes, occupancy */                                                        \
  dc_status prepare_kernel(int smem, int* blocks_per_sm);                                   \
  dc_status launch(const FxArgs& a, int grid, int smem, cudaStream_t s);

namespace f32 { DC_FX_DECLARE }
namespace f64 { DC_FX_DECLARE }
#undef DC_FX_DECLARE

}  // namespace fx
}  // namespace dc

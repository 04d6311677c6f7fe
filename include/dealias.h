/*
 * dealias.h -- C ABI of a GB300 (sm_103a) library for implicitly dealiased
 * linear convolutions, after J. C. Bowman and M. Roberts, "Efficient
 * Dealiased Convolutions without Padding", SIAM J. Sci. Comput. (2011).
 *
 * Every zero-padded DFT of size 2m, 3m or 4m is computed as q sub-transforms
 * of size m on residues of the padded index (Eqs. (2.1)-(2.2), Sec. 2.2,
 * Sec. 4.1); the padded array is never formed in device memory.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Arrays are row-major, last dimension contiguous (Sec. 3.1), complex values
 *   interleaved (re, im).  dtype DC_C64 = complex64 (float32 pairs) computed in
 *   FP32; DC_C128 = complex128 computed in FP64.  Root-of-unity tables are
 *   always generated in FP64 and rounded to the working precision.
 * - f, g, e, w, h, df, dg and work are DEVICE pointers owned by the caller; the
 *   library never frees them.  They must be aligned to the element size
 *   (8 bytes for DC_C64, 16 for DC_C128), else DC_ERR_ALIGN.  An output may be
 *   the same pointer as an input (in place, as in the paper); any other
 *   overlap is DC_ERR_ARG.
 * - work is caller-provided device scratch of at least the size that
 *   dc_workspace_size (or dc_batched_plan_workspace_size) reports, aligned to
 *   256 bytes; its first 256 bytes hold a device status word.  Two calls that
 *   may run concurrently must not share a workspace.
 * - stream is a cudaStream_t (NULL = legacy default stream).  Calls enqueue
 *   work and return; argument errors are detected on the host and returned
 *   synchronously, before anything is enqueued.  Errors found by kernels are
 *   recorded in the workspace status word, read with dc_read_status.
 * - Sizes: every transform length must be 2^a 3^b 5^c (any a, b, c >= 0; odd
 *   Hermitian m = 2c+1 included, Sec. 2.3).  A length whose factors include
 *   both 3 and 5 runs as direct DFTs up to 512, and above that when it splits
 *   into two factors with one odd prime each (e.g. 720 = 20 x 36); lengths
 *   without a plan, and lengths with another prime factor, return
 *   DC_ERR_SIZE (dc_workspace_size reports which).  The first call for a new
 *   size builds that size's root tables with cudaMalloc and a generator
 *   kernel; to keep allocation out of a captured CUDA graph, call dc_prepare
 *   first.
 * - Thread safety: calls may come from several host threads; table creation
 *   is serialized inside the library.
 */
#ifndef DEALIAS_H
#define DEALIAS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t dc_status;
#define DC_OK          0
#define DC_ERR_ARG     1  /* null pointer, bad dtype/kind, negative size, bad overlap */
#define DC_ERR_SIZE    2  /* size not 2^a 3^b 5^c, without a plan, or too large */
#define DC_ERR_ALIGN   3  /* pointer not aligned to its element size / workspace to 256 */
#define DC_ERR_CUDA    4  /* a CUDA runtime call failed (dc_last_cuda_error gives it) */
#define DC_ERR_TIMEOUT 5  /* a bounded device-side wait ran out (device status word) */
#define DC_ERR_NOMEM   6  /* workspace smaller than the size the query reports */
#define DC_ERR_DEVICE  7  /* a kernel's own consistency check failed (device status) */

#define DC_C64  0
#define DC_C128 1

#define DC_KIND_COMPLEX           0
#define DC_KIND_HERMITIAN         1
#define DC_KIND_TERNARY           2
#define DC_KIND_COMPLEX_ADJOINT   3
#define DC_KIND_HERMITIAN_ADJOINT 4
#define DC_KIND_COMPLEX_DOT2      5  /* f1 * g1 + f2 * g2, complex (dc_conv_complex_dot2) */
#define DC_KIND_HERMITIAN_DOT2    6  /* f1 * g1 + f2 * g2, centered Hermitian (dc_conv_hermitian_dot2) */

/* Human-readable name of a status code (static string). */
const char* dc_status_string(dc_status s);

/* cudaError_t value of the most recent DC_ERR_CUDA on this host thread. */
int32_t dc_last_cuda_error(void);

/* Workspace bytes a call of `kind` on the unpadded sizes dims[0..ndim-1] needs.
 * dims are the unpadded sizes m per dimension (for Hermitian kinds, the
 * centered dimensions are given as m, not 2m-1).  DC_ERR_SIZE/ARG as above. */
dc_status dc_workspace_size(int32_t kind, int32_t ndim, const int64_t* dims, int32_t dtype,
                            size_t* bytes);

/* 3D calls (Sec. 3.4) run the x-level residue slabs through their (y, z) work
 * arrays a chunk of slabs at a time, reusing the work arrays chunk after
 * chunk (the decoupled work arrays of Sec. 1 and Sec. 3.1).  The chunk size
 * follows the workspace the caller passes: the size dc_workspace_size reports
 * holds the default chunk (about 512 MB of work arrays); a smaller workspace
 * gives smaller chunks, down to one slab (3 m_x slabs for Hermitian kinds,
 * 2 m_x for complex ones), with the same result.
 * dc_workspace_size_slabs: workspace bytes of a 3D call of `kind` on dims
 * (ndim must be 3) whose chunks hold at most slabs_per_chunk (>= 1) slabs;
 * slabs_per_chunk = 1 gives the smallest workspace a 3D call accepts.
 * dc_chunking: the chunking a call of `kind` on dims makes with work_bytes of
 * workspace: *slabs_per_chunk and *chunks (the last chunk holds the rest);
 * *chunks = 0 when the workspace is too small for any call (which then
 * returns DC_ERR_NOMEM).  2D calls have one pass: *slabs_per_chunk = 0 and
 * *chunks = 1 when work_bytes suffices.  DC_ERR_ARG / DC_ERR_SIZE as above. */
dc_status dc_workspace_size_slabs(int32_t kind, int32_t ndim, const int64_t* dims, int32_t dtype,
                                  int64_t slabs_per_chunk, size_t* bytes);
dc_status dc_chunking(int32_t kind, int32_t ndim, const int64_t* dims, int32_t dtype, size_t work_bytes,
                      int64_t* slabs_per_chunk, int64_t* chunks);

/* Builds the root tables for a call of `kind` on dims (allocates device
 * memory once per size and device).  Optional; the first call does it too. */
dc_status dc_prepare(int32_t kind, int32_t ndim, const int64_t* dims, int32_t dtype);

/* Copies the workspace status word to the host after synchronizing `stream`.
 * *status = DC_OK or the first error a kernel recorded since the workspace
 * was last cleared by an entry point; *detail = kernel-specific detail. */
dc_status dc_read_status(const void* work, void* stream, int32_t* status, int32_t* detail);

/* Trace counters of the last batched launch on the fixed-shape engine
 * (workspace header), after synchronizing `stream`; no counterpart in the
 * paper.  out[0] = tasks that found their dependency unmet, out[1] = SM
 * cycles they waited, out[2..5] = SM cycles spent in level-1 tasks and in
 * the tasks of passes A, B, C, out[6..9] = the number of such tasks,
 * out[10] = SM cycles between the end of a task and the start of the next
 * (queue, dependency check), out[11] = SM cycles spent loading root tables
 * (12 entries).  Other kernels leave them zero. */
dc_status dc_read_trace(const void* work, void* stream, uint64_t* out);

/* ---------------------------------------------------------------------------
 * 1D complex binary convolution (Sec. 2.1, Eqs. (2.1)-(2.2), Function cconv).
 * f, g: m complex values, Fourier origin at index 0.  Writes the dealiased
 * linear convolution h_k = sum_{p=0}^{k} f_p g_{k-p}, k = 0..m-1 (N = 2m).
 * ------------------------------------------------------------------------- */
dc_status dc_conv_complex_1d(const void* f, const void* g, void* h, int64_t m, int32_t dtype,
                             void* work, size_t work_bytes, void* stream);

/* General implicit padding (Sec. 2.4): 1D complex convolution of f and g,
 * each holding p m values (wavenumbers 0..pm-1), implicitly zero padded to
 * N = q m.  The padded transform of size q m is computed as q transforms of
 * size m of the p-term sums W_r(s) = sum_{t<p} zeta_{qm}^{r(tm+s)} U_{tm+s}
 * (r < q), and the forward transform as q transforms of size m read at
 * k mod m for every output.  Writes h_k = sum_j F_j G_{(k-j) mod qm},
 * k = 0..nout-1, the cyclic convolution of the zero-padded inputs: for
 * q >= 2p the outputs k < 2pm - 1 are the full linear convolution
 * sum_{j} f_j g_{k-j} (p = 1, q = 2, nout = 2m - 1: all 2m - 1 outputs of the
 * linear convolution of Sec. 2.1, of which dc_conv_complex_1d returns the
 * first m) and the rest are zero; for q < 2p they wrap modulo qm.
 * 1 <= p <= q <= 16, 1 <= nout <= q m; m of the form 2^a 3^b 5^c with a
 * shared-memory transform (m up to several thousand), q m <= 2^24.  f, g:
 * p m values, h: nout values; h may be f or g (in place) when that array
 * holds nout values, no other overlap.  Workspace: dc_workspace_size_pq
 * bytes.  DC_ERR_ARG for p, q or nout out of range; DC_ERR_SIZE for an m
 * without such a transform. */
dc_status dc_workspace_size_pq(int64_t m, int32_t p, int32_t q, int64_t nout, int32_t dtype, size_t* bytes);
dc_status dc_conv_complex_1d_pq(const void* f, const void* g, void* h, int64_t m, int32_t p, int32_t q,
                                int64_t nout, int32_t dtype, void* work, size_t work_bytes, void* stream);

/* 1D centered Hermitian convolution under the 2/3 rule (Sec. 2.3, Function
 * conv; N = 3m).  f, g hold the wavenumbers 0..m-1 of Hermitian data
 * (U_{-k} = conj U_k); f_0 is taken as Re f_0 (Hermitian symmetry enforced,
 * Sec. 5).  h_k = sum_{p=k-m+1}^{m-1} f_p g_{k-p}, k = 0..m-1.  Any m of
 * the allowed form, odd or even: the sub-transforms are full complex
 * transforms of w^f + i w^g, so the odd case m = 2c+1 (which the paper leaves
 * undocumented) needs no special treatment. */
dc_status dc_conv_hermitian_1d(const void* f, const void* g, void* h, int64_t m, int32_t dtype,
                               void* work, size_t work_bytes, void* stream);

/* 1D centered Hermitian ternary convolution (Sec. 4.2, Function tconv;
 * N = 4m).  h_k = sum_{p+q+r=k} f_p g_q e_r over p,q,r in [-m+1, m-1],
 * k = 0..m-1; inputs as for dc_conv_hermitian_1d (any m of the allowed form). */
dc_status dc_conv_ternary_hermitian_1d(const void* f, const void* g, const void* e, void* h,
                                       int64_t m, int32_t dtype, void* work, size_t work_bytes,
                                       void* stream);

/* Gradients (no counterpart in the paper; defined for the real loss
 * L = Re sum_k conj(w_k) h_k with grad = dL/dRe x + i dL/dIm x):
 * complex:   df_p = sum_{k>=p} w_k conj(g_{k-p}),  dg_q = sum_{k>=q} w_k conj(f_{k-q}),
 *            computed by the same N = 2m residue machinery with the product
 *            W^ conj(G^) (a correlation with the conjugate partner).
 * Hermitian: df = S * conv_hermitian(W, g), dg = S * conv_hermitian(W, f),
 *            where W = w except W_0 = 2 Re w_0 and S halves index 0.
 * w, f, g are inputs; df, dg outputs (m values each). */
dc_status dc_conv_complex_1d_adjoint(const void* w, const void* f, const void* g, void* df,
                                     void* dg, int64_t m, int32_t dtype, void* work,
                                     size_t work_bytes, void* stream);
dc_status dc_conv_hermitian_1d_adjoint(const void* w, const void* f, const void* g, void* df,
                                       void* dg, int64_t m, int32_t dtype, void* work,
                                       size_t work_bytes, void* stream);

/* dc_conv_complex_1d without a workspace (no counterpart in the paper).
 * Same arguments and result as dc_conv_complex_1d, minus work/work_bytes.
 * For callers that cannot allocate device memory: code that runs under a CUDA
 * stream capture in global mode (cudaMalloc is prohibited there), code whose
 * device memory belongs to an allocator it may not bypass, and real-time loops
 * that cannot afford cudaMalloc's implicit synchronization.  It calls no
 * cudaMalloc, cudaFree or allocating routine: its scratch is one fixed 2 MiB
 * device array inside the library, held by every GPU that loads the library
 * until the process exits.  Limit: m <= 40960 for DC_C64 and m <= 20480 for
 * DC_C128; larger m returns DC_ERR_SIZE.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  All calls share
 * the one array, and each call rebuilds its root table and clears its status
 * word there, so calls whose GPU work may overlap (different streams, or
 * concurrent host threads) race and must be serialized by the caller. */
dc_status dc_conv_complex_1d_noalloc(const void* f, const void* g, void* h, int64_t m,
                                     int32_t dtype, void* stream);

/* ---------------------------------------------------------------------------
 * 2D and 3D convolutions (Sec. 3).  Layout row-major, last axis contiguous.
 * Complex (Functions cconv2, cconv3; N = 2m per axis): f, g, h of shape
 *   (mx, my) or (mx, my, mz); h_k = sum_{0<=p<=k} f_p g_{k-p} componentwise.
 * Centered Hermitian (Function conv2 and the 3D analogue; N = 3m per axis):
 *   shape (2mx-1, my) or (2mx-1, 2my-1, mz); the leading axes are centered
 *   (index i <-> wavenumber i - (m-1)), the last axis holds wavenumbers
 *   0..m-1 and U_{-k} = conj U_k for the whole wave vector.  The last-axis-0
 *   row (2D) / plane (3D) is projected onto that symmetry before convolving
 *   (U(k',0) <- (U(k',0) + conj U(-k',0))/2, Sec. 5); inputs are not modified.
 *   h_k = sum_p f_p g_{k-p} over p with |p_d|, |k_d - p_d| <= m_d - 1.
 * Gradients as for 1D (same loss convention); for Hermitian data the
 *   upstream array is symmetrized on the last-axis-0 row/plane,
 *   W(k',0) = w(k',0) + conj w(-k',0), and the outputs are halved there.
 * dims: mx, my (, mz) are the unpadded sizes (for Hermitian, m not 2m-1).
 * ------------------------------------------------------------------------- */
dc_status dc_conv_complex_2d(const void* f, const void* g, void* h, int64_t mx, int64_t my,
                             int32_t dtype, void* work, size_t work_bytes, void* stream);
dc_status dc_conv_complex_3d(const void* f, const void* g, void* h, int64_t mx, int64_t my,
                             int64_t mz, int32_t dtype, void* work, size_t work_bytes, void* stream);
dc_status dc_conv_hermitian_2d(const void* f, const void* g, void* h, int64_t mx, int64_t my,
                               int32_t dtype, void* work, size_t work_bytes, void* stream);
dc_status dc_conv_hermitian_3d(const void* f, const void* g, void* h, int64_t mx, int64_t my,
                               int64_t mz, int32_t dtype, void* work, size_t work_bytes,
                               void* stream);
/* 2D and 3D centered Hermitian ternary convolutions (Sec. 4; Function tconv2
 * and its 3D analogue): inputs f, g, e and output h of the Hermitian layout
 * above; h_k = sum_{p+q+r=k} f_p g_q e_r over p, q, r in the box
 * |p_d| <= m_d - 1 (componentwise), for the stored k.  Every axis is padded
 * implicitly to N = 4m: the outer (centered) axes with the leading zero
 * U_{-m} and two residues of 2m-point sub-transforms (Sec. 4.1, Procedures
 * fft0tpadBackward / fft0tpadForward, Eqs. (fft0tbackward)-(fft0tforward)),
 * the last axis by the 1D ternary rows (Sec. 4.2, Function tconv).  Inputs
 * are projected on the last-axis-0 row / plane as for the binary case. */
dc_status dc_conv_ternary_hermitian_2d(const void* f, const void* g, const void* e, void* h, int64_t mx,
                                       int64_t my, int32_t dtype, void* work, size_t work_bytes, void* stream);
dc_status dc_conv_ternary_hermitian_3d(const void* f, const void* g, const void* e, void* h, int64_t mx,
                                       int64_t my, int64_t mz, int32_t dtype, void* work, size_t work_bytes,
                                       void* stream);
dc_status dc_conv_complex_2d_adjoint(const void* w, const void* f, const void* g, void* df,
                                     void* dg, int64_t mx, int64_t my, int32_t dtype, void* work,
                                     size_t work_bytes, void* stream);
dc_status dc_conv_complex_3d_adjoint(const void* w, const void* f, const void* g, void* df,
                                     void* dg, int64_t mx, int64_t my, int64_t mz, int32_t dtype,
                                     void* work, size_t work_bytes, void* stream);
dc_status dc_conv_hermitian_2d_adjoint(const void* w, const void* f, const void* g, void* df,
                                       void* dg, int64_t mx, int64_t my, int32_t dtype, void* work,
                                       size_t work_bytes, void* stream);
dc_status dc_conv_hermitian_3d_adjoint(const void* w, const void* f, const void* g, void* df,
                                       void* dg, int64_t mx, int64_t my, int64_t mz, int32_t dtype,
                                       void* work, size_t work_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Inputs as arrays of vectors (Sec. 3, "2D pseudospectral application"): the
 * product f * g read as the dot product of two pairs,
 *   h = f1 * g1 + f2 * g2,
 * with * the complex convolution (Functions cconv, cconv2, cconv3) or the
 * centered Hermitian convolution (Functions conv, conv2 and the 3D
 * analogue).  The two pointwise products are summed in physical space, so
 * per residue one forward transform serves both pairs: five transforms per
 * residue for the complex kind instead of six, and, with the real transforms
 * of each Hermitian pair sharing one complex transform, three instead of
 * four for the Hermitian kind.  The advective term of the 2D Euler equation,
 * u . grad w, is dc_conv_hermitian_dot2 of (i k_x w, i k_y w) with
 * (i k_y w / k^2, -i k_x w / k^2).
 * ndim = 1, 2 or 3; dims: the unpadded sizes as for the single-pair calls;
 * f1, g1, f2, g2, h: device arrays of the single-pair layout; h may be any
 * of the inputs (in place); each Hermitian input is projected as for the
 * single-pair call.  Workspace: dc_workspace_size with DC_KIND_*_DOT2 (3D:
 * chunks follow the workspace as for the single-pair calls).
 * ------------------------------------------------------------------------- */
dc_status dc_conv_complex_dot2(int32_t ndim, const int64_t* dims, const void* f1, const void* g1,
                               const void* f2, const void* g2, void* h, int32_t dtype, void* work,
                               size_t work_bytes, void* stream);
dc_status dc_conv_hermitian_dot2(int32_t ndim, const int64_t* dims, const void* f1, const void* g1,
                                 const void* f2, const void* g2, void* h, int32_t dtype, void* work,
                                 size_t work_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Batched 1D complex convolutions of uneven sizes in one persistent launch.
 * A plan fixes the sizes m[0..n-1] (host array), the dtype and the per-size
 * kernel configuration; instance i occupies elements [off_i, off_i + m_i) of
 * the packed arrays f, g, h with off_i = m_0 + ... + m_{i-1}.
 * When every m lies in {2^a, 3*2^a, 5*2^a}, 64 <= m <= 65536, the plan runs
 * on the fixed-shape engine (compile-time code per size; instances with
 * m <= 256 E wholly in shared memory, larger ones as row/column passes
 * through L2-resident scratch, all as tasks of one persistent queue);
 * otherwise on the runtime-shaped engine.
 * flags: DC_PLAN_AUTOTUNE = time candidates on the current device (the queue
 * order of the fixed-shape engine, the per-size configuration of the
 * runtime-shaped one; needs the GPU idle), DC_PLAN_ONE_PER_LAUNCH = one
 * launch per instance, in instance order (the "plain" comparison mode).
 * Planning allocates device memory; execution does not.
 * dc_conv_complex_1d_batched may be captured in a CUDA graph.
 * ------------------------------------------------------------------------- */
typedef struct dc_batched_plan dc_batched_plan;
#define DC_PLAN_AUTOTUNE        1
#define DC_PLAN_ONE_PER_LAUNCH  4
dc_status dc_batched_plan_create(const int64_t* m, int32_t n, int32_t dtype, int32_t flags,
                                 dc_batched_plan** plan);
dc_status dc_batched_plan_workspace_size(const dc_batched_plan* plan, size_t* bytes);
/* Number of kernel launches one execution of the plan issues. */
dc_status dc_batched_plan_launches(const dc_batched_plan* plan, int32_t* launches);
/* Configuration chosen for the i-th distinct size of the plan (sizes in
 * increasing order): *level 1 = whole sub-transform in shared memory with *nt
 * instances per block, 2 = two-level m = l1 * l2 through scratch with column
 * tiles of width *w.  Any output pointer may be NULL.  DC_ERR_ARG if i is out
 * of range. */
dc_status dc_batched_plan_describe(const dc_batched_plan* plan, int32_t i, int64_t* m,
                                   int32_t* level, int32_t* nt, int32_t* l1, int32_t* l2,
                                   int32_t* w);
/* Queue order of a plan on the fixed-shape engine (every size in the set
 * {2^a, 3*2^a, 5*2^a}, 64 <= m <= 65536; not the one-per-launch mode): *batch_target = column tiles
 * per batch of two-level instances (the pipeline distance between their
 * passes), *l1_mode = placement of the one-level work (0 after the
 * two-level pipeline, 1 the larger half spread over it, 2 before it).  No
 * counterpart in the paper (a GPU scheduling choice).  DC_ERR_ARG for other
 * plans. */
dc_status dc_batched_plan_schedule(const dc_batched_plan* plan, int32_t* batch_target,
                                   int32_t* l1_mode);
/* Rebuilds the queue of such a plan with the given order (batch_target >= 1,
 * 0 <= l1_mode <= 2); the result does not depend on it, only the time does.
 * The workspace size may change: query it again.  Not while a launch of the
 * plan is in flight.  DC_ERR_ARG for other plans or values. */
dc_status dc_batched_plan_set_schedule(dc_batched_plan* plan, int32_t batch_target, int32_t l1_mode);
/* Column tiles (passes A, C) or row groups (pass B) each task of such a plan
 * runs, 1 to 4 (no counterpart in the paper: fewer, longer tasks spend less
 * of the launch handing over between tasks, more keep the blocks balanced).
 * DC_PLAN_AUTOTUNE picks it with the queue order; _set_ rebuilds the queue
 * with the given value (same result, other timing; query the workspace size
 * again; not while a launch of the plan is in flight).  DC_ERR_ARG for other
 * plans or values. */
dc_status dc_batched_plan_task_units(const dc_batched_plan* plan, int32_t* units);
dc_status dc_batched_plan_set_task_units(dc_batched_plan* plan, int32_t units);
/* Split variants of the two-level sizes of such a plan (FP32 plans; no
 * counterpart in the paper: a tile-shape choice of this engine).  A size m of
 * the set above 2^12 (3*2^11, 5*2^10) runs its m-point sub-transforms as
 * L1-point rows and L2-point columns, m = L1 * L2; variant 0 takes L2 = 128
 * up to m = 32768 and 256 above, variant 1 takes L2 = 64 for 8192, 12288
 * and 10240 and the other of 128 and 256 for the rest, which changes the
 * row length, the threads per row and the column tile width.
 * Bit c of *mask is set when the size with size code c (the position of m
 * in 64, 128, ..., 65536, 96, ..., 49152, 80, ..., 40960) runs variant 1;
 * dc_batched_plan_describe reports the resulting L1, L2 and tile width.
 * DC_PLAN_AUTOTUNE times both variants of every such size of the plan on
 * that size's instances alone and keeps variant 1 where it is faster by at
 * least 1 %.  _set_ rebuilds the queue with the given mask (bits of sizes
 * without a second variant, and every bit of FP64 plans, are ignored; the
 * result does not depend on it, only the time does; query the workspace
 * size again; not while a launch of the plan is in flight).  DC_ERR_ARG for
 * plans off the fixed-shape engine or in the one-per-launch mode. */
dc_status dc_batched_plan_variants(const dc_batched_plan* plan, uint32_t* mask);
dc_status dc_batched_plan_set_variants(dc_batched_plan* plan, uint32_t mask);
dc_status dc_conv_complex_1d_batched(const dc_batched_plan* plan, const void* f, const void* g,
                                     void* h, void* work, size_t work_bytes, void* stream);
/* Failure-path self-test, no counterpart in the paper: launches the
 * fixed-shape batched kernel on a one-task queue whose dependency counter
 * nothing advances, with a wait limit of `cycles` SM cycles.  The task's
 * bounded wait runs out and the kernel records DC_ERR_TIMEOUT (detail: the
 * task index, 0) in the status word of `work` (>= 1024 bytes, 256-aligned,
 * device memory), readable with dc_read_status after the stream completes.
 * Nothing faults or hangs.  DC_ERR_ARG / ALIGN / NOMEM on bad arguments. */
dc_status dc_selftest_wait_timeout(void* work, size_t work_bytes, int64_t cycles, void* stream);
/* End-to-end batched convolution from host memory (no counterpart in the
 * paper: a transfer schedule).  The instances are split into `nchunks`
 * chunks of consecutive instances with about equal element counts; chunk k's
 * slices of hf, hg are copied into df, dg, its convolutions run as soon as
 * they have arrived, and its results are copied from dh back to hh, each
 * step on library streams, so that copies in both directions overlap
 * the computation of other chunks.  The streams start after the work
 * already enqueued on `stream`, and `stream` continues after all of it.
 * hf, hg, hh: host arrays of the packed layout (page-locked for the copies
 * to overlap); df, dg, dh: device arrays of the same size; work: device
 * workspace of dc_batched_plan_host_workspace_size bytes for this nchunks.
 * The first call for a given nchunks plans the chunks (device allocation;
 * call dc_batched_plan_host_workspace_size first to keep it out of a
 * captured graph).  Results equal dc_conv_complex_1d_batched's. */
dc_status dc_batched_plan_host_workspace_size(dc_batched_plan* plan, int32_t nchunks, size_t* bytes);
dc_status dc_conv_complex_1d_batched_host(dc_batched_plan* plan, const void* hf, const void* hg, void* hh,
                                          void* df, void* dg, void* dh, void* work, size_t work_bytes,
                                          int32_t nchunks, void* stream);
dc_status dc_batched_plan_destroy(dc_batched_plan* plan);

/* Partition of a batch of independent 1D convolutions across nranks
 * processes (one per GPU) by the longest-processing-time rule: instances
 * in order of decreasing cost m log2 m (the sub-transforms' operation count,
 * Sec. 2.1), equal costs in instance order, each to the rank with the least
 * load so far (ties: the lowest rank).  No counterpart in the paper (a
 * scheduling choice for running one batch on several GPUs, each rank then
 * planning and convolving its own instances with no exchange of data).
 * m: n sizes (host, >= 1).  owner: n ranks written (host).  load: nranks
 * summed costs written (host), or NULL.  Host code only: needs no GPU.
 * DC_ERR_ARG for n < 0, nranks < 1, a size < 1 or a NULL array with n > 0. */
dc_status dc_partition_lpt(const int64_t* m, int32_t n, int32_t nranks, int32_t* owner, double* load);

#ifdef __cplusplus
}
#endif

#endif /* DEALIAS_H */

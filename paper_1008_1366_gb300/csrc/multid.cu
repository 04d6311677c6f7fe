// 2D and 3D implicitly dealiased convolutions (Sec. 3) composed from the
// outer-axis passes (axis.cu) and the batched row kernels (conv1d.cuh).
//
//   2D (Functions cconv2, conv2): x-backward of each input into q_x residue
//     arrays (m_x rows each) -> one 1D convolution along y per row of every
//     residue array (in place) -> x-forward recombining the residues.
//   3D (Function cconv3 and the centered Hermitian analogue): x-backward ->
//     for every x-row slab a 2D convolution in (y, z), itself y-backward ->
//     rows along z -> y-forward written back into the slab -> x-forward.
// The (y, z) work arrays are decoupled from the data, as the paper stresses
// (Sec. 1, Sec. 3.1): slabs are processed in chunks whose work arrays fit in
// a fixed budget and are reused chunk after chunk.  The budget is sized for
// full launches, not for L2: each chunk runs three launches (y-backward,
// rows, y-forward) whose last wave of blocks is partly idle, and at 256^3
// fewer, larger chunks gained more than keeping a chunk in L2 (forward
// call, budget 64 / 128 / 256 / 512 MB: 6.60 / 6.21 / 5.89 / 5.63 ms).
// Gradients use the same composition with three transformed inputs
// (w, f, g) and the gradient row kernels; for Hermitian data the upstream
// array is symmetrized on the self-conjugate subspace on load and the outputs
// halved there on store.
#include <algorithm>

#include "conv1d.cuh"
#include "fixed.h"
#include "launch.h"
#include "multid.h"
#include "plan.h"
#include "tables.h"

namespace dc {
namespace {

// the fixed engine's kind for a row kind, -1 where it has none
int row_mode(int row_kind) {
  switch (row_kind) {
    case K_COMPLEX: return fx::MODE_COMPLEX;
    case K_HERMITIAN: return fx::MODE_HERM;
    case K_HERMITIAN_PAIR: return fx::MODE_PAIR;
    case K_HERMITIAN_DOT2: return fx::MODE_HDOT2;
  }
  return -1;
}

constexpr size_t kHeader = sizeof(WorkHeader);
constexpr size_t kChunkBudget = 512ull << 20;   // bytes of (y, z) work arrays per chunk

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Md {
  int pk = 0, ndim = 0, ds = 0;
  int64_t m[3] = {0, 0, 0};
  bool herm = false, adj = false, tern = false;
  int64_t Lx = 0, Ly = 0;     // sub-transform lengths of the outer axes (m, or 2m for ternary)
  int qa = 2, narr = 2, nout = 1, row_kind = K_COMPLEX;
  int64_t ny_in = 0;          // stored y extent (3D): my or 2my-1
  int64_t nx = 0;             // elements of one x-level residue array
  int64_t slabs = 0, sx = 0;  // 3D: slabs and elements per slab
  int64_t S = 0;              // 3D: slabs per chunk
  AxisArgs ax, ay;            // outer-axis templates (plan, tile width, table)
  CfgDev rows;                // row configuration
  bool rows_fx = false;       // rows on the fixed-shape engine
  int rows_mode = -1;         // its kind of convolution (fx::MODE_*)
  int64_t rows_n[2] = {0, 0}; // row counts of the row launches (full chunk, last chunk)
  int rows_grid = 1;
  size_t rows_slot = 0;
  size_t off_y = 0, off_rows = 0, total = 0;
};

int smem_cap() { return device_info().smem_optin - kStaticSmemReserve; }

// mode: 0 complex, 1 centered (q = 3), 2 centered ternary (q = 2, length
// 2m), 3 centered ternary (q = 4, length m)
bool axis_cfg(int mode, int64_t m, int ds, bool with_table, AxisArgs* a) {
  const int emax = ds == 8 ? 30 : 15;
  FftPlan p;
  const int64_t L = mode == 2 ? 2 * m : m;
  if (m < 1 || L > (1 << 16) || !make_fft_plan((int)L, emax, &p)) return false;
  if (p.tpt > 512) return false;
  const int colb = axis_smem(true, mode, (int)m, 1, ds);
  int w = 1;
  while (w * 2 <= 32 && (w * 2) * p.tpt <= 512 && (w * 2) * colb <= smem_cap()) w *= 2;
  if (colb > smem_cap()) return false;
  *a = AxisArgs{};
  a->m = (int32_t)m;
  a->centered = mode;
  a->w = w;
  a->p = p;
  a->TN = (int32_t)((mode >= 2 ? 4 : mode == 1 ? 3 : 2) * m);
  if (with_table) {
    const void* tw = nullptr;
    if (get_root_table(a->TN, ds, &tw) != DC_OK) return false;
    a->tw = tw;
  }
  return true;
}

// slabs_req > 0 (3D only): run the (y, z) work arrays for at most that many
// x-slabs per chunk instead of the default budget's count.
dc_status plan_md(int pk, int ndim, const int64_t* dims, int ds, bool with_tables, Md* md,
                  int64_t slabs_req = 0) {
  if (ndim < 2 || ndim > 3) return DC_ERR_ARG;
  for (int d = 0; d < ndim; ++d) {
    if (dims[d] < 1) return DC_ERR_ARG;
    md->m[d] = dims[d];
  }
  md->pk = pk; md->ndim = ndim; md->ds = ds;
  const bool dot = pk == DC_KIND_COMPLEX_DOT2 || pk == DC_KIND_HERMITIAN_DOT2;
  md->tern = pk == DC_KIND_TERNARY;
  md->herm = pk == DC_KIND_HERMITIAN || pk == DC_KIND_HERMITIAN_ADJOINT || pk == DC_KIND_HERMITIAN_DOT2 || md->tern;
  md->adj = pk == DC_KIND_COMPLEX_ADJOINT || pk == DC_KIND_HERMITIAN_ADJOINT;
  if (pk < 0 || pk > DC_KIND_HERMITIAN_DOT2) return DC_ERR_ARG;
  // outer axes: centered for Hermitian data; for the ternary kind N = 4m
  // per axis (Sec. 4.1), as four m-point residues where the compile-time
  // axis kernels take every outer length (the residue inputs fold U_k and
  // U_{k-m} like the centered case, with zeta_4 for zeta_3), else as two
  // residues of 2m points
  const bool tern4 = md->tern && fixed_axis_len(dims[0]) && (ndim == 2 || fixed_axis_len(dims[1]));
  const int amode = md->tern ? (tern4 ? 3 : 2) : (md->herm ? 1 : 0);
  md->qa = axis_q(amode);
  md->narr = dot ? 4 : (md->adj || md->tern ? 3 : 2);
  md->nout = md->adj ? 2 : 1;
  md->row_kind = md->tern ? K_TERNARY
                 : dot ? (md->herm ? K_HERMITIAN_DOT2 : K_COMPLEX_DOT2)
                       : md->herm ? (md->adj ? K_HERMITIAN_PAIR : K_HERMITIAN)
                                  : (md->adj ? K_COMPLEX_ADJ : K_COMPLEX);
  const int64_t mx = md->m[0], my = md->m[1], mlast = md->m[ndim - 1];
  md->Lx = axis_len(amode, (int)mx);
  md->Ly = ndim == 3 ? axis_len(amode, (int)my) : 0;
  if (!axis_cfg(amode, mx, ds, with_tables, &md->ax)) return DC_ERR_SIZE;
  int64_t nrows;   // rows of the row kernel per launch
  if (ndim == 2) {
    md->nx = md->Lx * my;
    nrows = md->qa * md->Lx;
  } else {
    if (!axis_cfg(amode, my, ds, with_tables, &md->ay)) return DC_ERR_SIZE;
    md->ny_in = md->herm ? 2 * my - 1 : my;
    md->nx = md->Lx * md->ny_in * mlast;
    md->slabs = md->qa * md->Lx;
    md->sx = md->ny_in * mlast;
    const size_t per_slab = (size_t)md->narr * md->qa * md->Ly * mlast * ds;
    md->S = std::max<int64_t>(1, std::min<int64_t>(md->slabs, kChunkBudget / per_slab));
    if (slabs_req > 0) md->S = std::min<int64_t>(slabs_req, md->slabs);
    nrows = md->qa * md->S * md->Ly;
  }
  if (!make_cfg(md->row_kind, mlast, ds, kThreads, smem_cap(), 0, &md->rows)) return DC_ERR_SIZE;
  if (with_tables) {
    const void* tw = nullptr;
    dc_status st = get_root_table(md->rows.TN, ds, &tw);
    if (st != DC_OK) return st;
    md->rows.tw = tw;
  }
  int bps = 1;
  if (with_tables) {
    dc_status st = conv1d_blocks_per_sm(md->row_kind, ds, md->rows.smem, &bps);
    if (st != DC_OK) return st;
  }
  const int64_t nitems = (nrows + md->rows.nt - 1) / md->rows.nt;
  md->rows_grid = (int)std::max<int64_t>(1, std::min<int64_t>(nitems, (int64_t)std::max(1, bps) * device_info().sms));
  if (!with_tables) md->rows_grid = (int)std::min<int64_t>(nitems, 4 * 1024);   // upper bound for sizing
  md->rows_slot = align_up(cfg_scratch_bytes(md->row_kind, md->rows, ds), 256);
  size_t off = kHeader + align_up((size_t)md->narr * md->qa * md->nx * ds, 256);
  md->off_y = off;
  if (ndim == 3) off += align_up((size_t)md->narr * md->qa * md->S * md->Ly * mlast * ds, 256);
  md->off_rows = off;
  size_t rows_bytes = (size_t)md->rows_grid * md->rows_slot;
  // binary complex and centered Hermitian rows of a size in the set, and
  // the gradient pair rows of a one-level size, run on the fixed-shape
  // engine
  md->rows_n[0] = nrows;
  md->rows_n[1] = ndim == 3 && md->slabs % md->S ? md->qa * (md->slabs % md->S) * md->Ly : nrows;
  // The gradient pair transforms W alone and keeps the real part of its
  // transform, which drops any non-Hermitian rounding of W's rows (two
  // plain convolutions with W packed beside g would carry it into g's
  // channel).
  md->rows_mode = row_mode(md->row_kind);
  md->rows_fx = fx_uniform_ok(mlast, ds) && md->rows_mode >= 0 &&
                ((md->rows_mode != fx::MODE_PAIR && md->rows_mode != fx::MODE_HDOT2) || !fx_uniform_two_level(mlast));
  // ternary rows of a one-level size of the set run on the fixed engine as
  // four m-point residues; those whose 2m-point sub-transforms are a
  // two-level size, on its two-residue ternary passes
  if (md->tern && fx_uniform_ok(mlast, ds) && !fx_uniform_two_level(mlast)) {
    md->rows_fx = true;
    md->rows_mode = fx::MODE_TERN4;
    rows_bytes = std::max(fx_uniform_work(md->rows_n[0], mlast, ds, md->rows_mode),
                          fx_uniform_work(md->rows_n[1], mlast, ds, md->rows_mode));
    if (with_tables) {
      for (int k = 0; k < 2; ++k) {
        dc_batched_plan* p = nullptr;
        dc_status st = fx_uniform_plan(md->rows_n[k], mlast, ds, &p, md->rows_mode);
        if (st != DC_OK) return st;
      }
    }
  } else if (md->tern && fx_ternary_ok(mlast, ds)) {
    md->rows_fx = true;
    md->rows_mode = fx::MODE_TERN;
    rows_bytes = std::max(fx_ternary_work(mlast, ds, md->rows_n[0]), fx_ternary_work(mlast, ds, md->rows_n[1]));
    if (with_tables) {
      for (int k = 0; k < 2; ++k) {
        dc_batched_plan* p = nullptr;
        dc_status st = fx_ternary_plan(mlast, ds, &p, md->rows_n[k]);
        if (st != DC_OK) return st;
      }
    }
  } else if (md->rows_fx) {
    rows_bytes = std::max(fx_uniform_work(md->rows_n[0], mlast, ds, md->rows_mode),
                          fx_uniform_work(md->rows_n[1], mlast, ds, md->rows_mode));
    if (with_tables) {
      for (int k = 0; k < 2; ++k) {
        dc_batched_plan* p = nullptr;
        dc_status st = fx_uniform_plan(md->rows_n[k], mlast, ds, &p, md->rows_mode);
        if (st != DC_OK) return st;
      }
    }
  }
  off += align_up(rows_bytes, 256);
  md->total = off;
  return DC_OK;
}

dc_status run_rows(const Md& md, const void* const* in, void* const* out, int64_t nrows, char* work,
                   cudaStream_t s) {
  if (md.rows_fx) {
    // the rows' own status header sits at the start of their region
    const int64_t m = md.m[md.ndim - 1];
    char* rw = work + md.off_rows;
    const size_t rb = md.total - md.off_rows;
    if (md.rows_mode == fx::MODE_TERN) return fx_ternary_run(m, md.ds, in[0], in[1], in[2], out[0], rw, rb, s, nrows);
    dc_batched_plan* p = nullptr;
    dc_status st = fx_uniform_plan(nrows, m, md.ds, &p, md.rows_mode);
    if (st != DC_OK) return st;
    if (md.rows_mode == fx::MODE_PAIR) return fx_pair_run(p, in[0], in[1], in[2], out[0], out[1], rw, rb, s);
    if (md.rows_mode == fx::MODE_HDOT2) return fx_hdot2_run(p, in[0], in[1], in[2], in[3], out[0], rw, rb, s);
    if (md.rows_mode == fx::MODE_TERN4) return fx_tern4_run(p, in[0], in[1], in[2], out[0], rw, rb, s);
    return dc_conv_complex_1d_batched(p, in[0], in[1], out[0], rw, rb, s);
  }
  ConvArgs a{};
  for (int x = 0; x < 4; ++x) a.in[x] = in[x];
  for (int o = 0; o < 2; ++o) a.out[o] = out[o];
  a.stride = md.m[md.ndim - 1];
  a.ninst = (int32_t)nrows;
  a.nitems = (int32_t)((nrows + md.rows.nt - 1) / md.rows.nt);
  a.hdr = (WorkHeader*)work;
  a.scratch = work + md.off_rows;
  a.slot_bytes = (int64_t)md.rows_slot;
  a.cfg0 = md.rows;
  const int grid = std::min(md.rows_grid, a.nitems);
  return launch_conv1d(md.row_kind, md.ds, a, grid, md.rows.smem, s);
}

}  // namespace

dc_status md_workspace(int pk, int ndim, const int64_t* dims, int ds, size_t* bytes) {
  Md md;
  dc_status st = plan_md(pk, ndim, dims, ds, false, &md);
  if (st == DC_OK) *bytes = md.total;
  return st;
}

dc_status md_workspace_slabs(int pk, int ndim, const int64_t* dims, int ds, int64_t slabs, size_t* bytes) {
  if (slabs < 1) return DC_ERR_ARG;
  Md md;
  dc_status st = plan_md(pk, ndim, dims, ds, false, &md, ndim == 3 ? slabs : 0);
  if (st == DC_OK) *bytes = md.total;
  return st;
}

// Slabs per chunk of a call given work_bytes of workspace: the default
// count when the workspace holds it, else the largest count whose
// workspace fits (the workspace grows with the count), 0 when not even one
// slab fits.
dc_status md_chunking(int pk, int ndim, const int64_t* dims, int ds, size_t work_bytes, int64_t* slabs,
                      int64_t* chunks) {
  Md md;
  dc_status st = plan_md(pk, ndim, dims, ds, false, &md);
  if (st != DC_OK) return st;
  if (ndim == 2) {
    *slabs = 0;
    *chunks = work_bytes >= md.total ? 1 : 0;
    return DC_OK;
  }
  int64_t S = 0;
  if (work_bytes >= md.total) {
    S = md.S;
  } else {
    int64_t lo = 1, hi = md.S - 1;
    while (lo <= hi) {
      const int64_t mid = lo + (hi - lo) / 2;
      Md t;
      if ((st = plan_md(pk, ndim, dims, ds, false, &t, mid)) != DC_OK) return st;
      if (t.total <= work_bytes) {
        S = mid;
        lo = mid + 1;
      } else {
        hi = mid - 1;
      }
    }
  }
  *slabs = S;
  *chunks = S ? (md.slabs + S - 1) / S : 0;
  return DC_OK;
}

dc_status md_prepare(int pk, int ndim, const int64_t* dims, int ds) {
  Md md;
  return plan_md(pk, ndim, dims, ds, true, &md);
}

dc_status md_run(int pk, int ndim, const int64_t* dims, int ds, const void* const* ins, int nin,
                 void* const* outs, int nout, void* work, size_t work_bytes, cudaStream_t s) {
  // 3D: the chunk of x-slabs whose (y, z) work arrays the workspace holds
  int64_t S = 0, nchunks = 0;
  dc_status st = md_chunking(pk, ndim, dims, ds, work_bytes, &S, &nchunks);
  if (st != DC_OK) return st;
  if (nchunks == 0) return DC_ERR_NOMEM;
  Md md;
  st = plan_md(pk, ndim, dims, ds, true, &md, S);
  if (st != DC_OK) return st;
  if (nin != md.narr || nout != md.nout) return DC_ERR_ARG;
  if (work_bytes < md.total) return DC_ERR_NOMEM;
  char* wk = (char*)work;
  char* X = wk + kHeader;
  const int64_t mx = md.m[0], my = md.m[1], mz = md.m[md.ndim - 1];
  const int qa = md.qa;
  auto xres = [&](int z, int r) { return (void*)(X + ((size_t)z * qa + r) * md.nx * ds); };
  // slot of gradient output o inside the transformed arrays (w, f, g): f -> df, g -> dg
  const int oslot0 = md.adj ? 1 : 0;
  DC_CUDA_TRY(cudaMemsetAsync(work, 0, kHeader, s));

  // x-backward
  AxisArgs ax = md.ax;
  ax.outer = 1;
  ax.inner = md.ndim == 2 ? my : md.ny_in * mz;
  ax.proj = md.herm ? md.ndim : 0;
  ax.proj_mz = mz;
  ax.proj_ny = md.ndim == 3 ? md.ny_in : 1;
  ax.dbl_mask = (pk == DC_KIND_HERMITIAN_ADJOINT) ? 1 : 0;
  for (int z = 0; z < md.narr; ++z) {
    ax.in[z] = ins[z];
    for (int r = 0; r < qa; ++r) ax.out[z * kAxisQ + r] = xres(z, r);
  }
  if ((st = launch_axis(false, ds, ax, md.narr, s)) != DC_OK) return st;

  if (md.ndim == 2) {
    const void* rin[4] = {nullptr, nullptr, nullptr, nullptr};
    void* rout[2] = {nullptr, nullptr};
    for (int z = 0; z < md.narr; ++z) rin[z] = xres(z, 0);
    for (int o = 0; o < md.nout; ++o) rout[o] = xres(oslot0 + o, 0);
    if ((st = run_rows(md, rin, rout, (int64_t)qa * md.Lx, wk, s)) != DC_OK) return st;
  } else {
    char* Y = wk + md.off_y;
    for (int64_t s0 = 0; s0 < md.slabs; s0 += md.S) {
      const int64_t Sc = std::min<int64_t>(md.S, md.slabs - s0);
      const size_t ych = (size_t)Sc * md.Ly * mz;   // elements of one y-level residue array
      auto yres = [&](int z, int r) { return (void*)(Y + ((size_t)z * qa + r) * ych * ds); };
      AxisArgs ay = md.ay;
      ay.outer = Sc;
      ay.inner = mz;
      for (int z = 0; z < md.narr; ++z) {
        ay.in[z] = X + ((size_t)z * qa * md.nx + (size_t)s0 * md.sx) * ds;
        for (int r = 0; r < qa; ++r) ay.out[z * kAxisQ + r] = yres(z, r);
      }
      if ((st = launch_axis(false, ds, ay, md.narr, s)) != DC_OK) return st;
      const void* rin[4] = {nullptr, nullptr, nullptr, nullptr};
      void* rout[2] = {nullptr, nullptr};
      for (int z = 0; z < md.narr; ++z) rin[z] = yres(z, 0);
      for (int o = 0; o < md.nout; ++o) rout[o] = yres(oslot0 + o, 0);
      if ((st = run_rows(md, rin, rout, (int64_t)qa * Sc * md.Ly, wk, s)) != DC_OK) return st;
      AxisArgs yf = md.ay;
      yf.outer = Sc;
      yf.inner = mz;
      for (int o = 0; o < md.nout; ++o) {
        for (int r = 0; r < qa; ++r) yf.fin[o * kAxisQ + r] = yres(oslot0 + o, r);
        yf.fout[o] = X + ((size_t)(oslot0 + o) * qa * md.nx + (size_t)s0 * md.sx) * ds;
      }
      if ((st = launch_axis(true, ds, yf, md.nout, s)) != DC_OK) return st;
    }
  }

  // x-forward
  AxisArgs xf = md.ax;
  xf.outer = 1;
  xf.inner = ax.inner;
  xf.proj = ax.proj;
  xf.proj_mz = ax.proj_mz;
  xf.proj_ny = ax.proj_ny;
  xf.halve_mask = (pk == DC_KIND_HERMITIAN_ADJOINT) ? 3 : 0;
  for (int o = 0; o < md.nout; ++o) {
    for (int r = 0; r < qa; ++r) xf.fin[o * kAxisQ + r] = xres(oslot0 + o, r);
    xf.fout[o] = outs[o];
  }
  return launch_axis(true, ds, xf, md.nout, s);
}

}  // namespace dc

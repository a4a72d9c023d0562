// Internal declarations shared by the host build, the kernels and the C ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "hbmc.h"

namespace hbmc {

// Every gathered device vector carries kGuard zero entries after its n_pad
// live entries; padded SELL slots point at index n_pad with value 0.
constexpr int64_t kGuard = 32;
constexpr int kMaxBs = 64;
constexpr int64_t kHistCap = 100000;

// Host-side result of hbmc_build: ordering, Abar and every packed layout.
struct HostLayout {
  int64_t n = 0, n_pad = 0, nnz = 0, nnz_lower = 0;
  int32_t bs = 1, w = 1, nc = 0;
  int64_t nblocks = 0, ntiles = 0;

  std::vector<int64_t> block_of;     // n
  std::vector<int32_t> block_color;  // nblocks
  std::vector<int64_t> pi;           // n: original -> padded HBMC index
  std::vector<int32_t> inv;          // n_pad: padded index -> original, -1 for dummies
  std::vector<int64_t> color_ptr;    // nc+1 (row index)
  std::vector<int64_t> tile_ptr;     // nc+1 (level-1 block index)

  // Abar = P A P^T, padded, sorted columns
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  std::vector<double> av;

  // strict lower part of Abar as CSR (IC(0) input) and its link to Abar
  std::vector<int64_t> lrp;
  std::vector<int32_t> lci;
  std::vector<double> laval;
  std::vector<int64_t> l_to_abar;  // lower entry -> position in Abar
  std::vector<double> adiag;       // n_pad

  // Nonsymmetric values (pattern still symmetric; ILU(0)): for lower entry
  // e = (i, j) the transposed value abar_ji and its position in Abar; the
  // upper triangle by rows (row i: columns j > i ascending, with the lower
  // entry (j, i) that carries u_ij).
  bool nonsym = false;
  std::vector<double> uaval;
  std::vector<int64_t> u_to_abar;
  std::vector<int64_t> urp, upos;
  std::vector<int32_t> uci;

  // SpMV: SELL with slice height w, column-major inside a slice
  std::vector<int64_t> a_ptr;  // nslices+1, entry offsets
  std::vector<int32_t> a_col;
  std::vector<double> a_val;

  // SpMV with long rows split (hbmc_options.sell_split): per slice a head
  // width; heads as SELL (sh_*); the cut-off pieces as rows of their own,
  // sorted by length, w to a slice (sp_*); the split rows in slice order with
  // their pieces' positions (cmb_*); per slice a lane mask of split rows and
  // the index of its first split row.
  int32_t split_piece = 0, split_cost = 0;
  std::vector<int32_t> split_head;
  std::vector<int64_t> sh_ptr, sp_ptr;
  std::vector<int32_t> sh_col, sp_col;
  std::vector<double> sh_val, sp_val;
  std::vector<uint32_t> sl_mask;
  std::vector<int32_t> sl_first, cmb_ptr, cmb_slot;
  int64_t split_rows = 0, split_pieces = 0;

  // SpMV with a variable slice height (hbmc_options.sell_vslice): per slice
  // of w rows its sub-slice height C and first sub-slice; per sub-slice its
  // start (the width is the length over C); entries column-major per sub-slice.
  int32_t vslice_cost = 0;
  std::vector<uint8_t> vs_c;
  std::vector<int64_t> vs_first, vs_ptr;
  std::vector<int32_t> vs_col;
  std::vector<double> vs_val;

  // Substitution layouts, one slice per (level-1 block, step).  "o" = entries
  // coupling to other colors (gathered from global memory), "i" = entries
  // coupling to earlier (forward) / later (backward) steps of the same BMC
  // block, addressed by step index m.
  std::vector<int64_t> fo_ptr, fi_ptr, bo_ptr, bi_ptr;  // nslices+1 each
  std::vector<int32_t> fo_col, bo_col;
  std::vector<uint8_t> fi_m, bi_m;
  // lower entry e -> slot of l_ij in the forward layout (>= 0: fo slot,
  // < 0: fi slot -v-1) and in the backward layout (bo / bi likewise)
  std::vector<int64_t> lmap_f, lmap_b;

  // The other-color entries again, without slice padding, for the
  // loader-thread sweeps: per level-1 block its rows one after another (row
  // lr = step * w + lane; each row's entries in the order of fo / bo), the
  // block's run padded to a multiple of 32 entries.  x_ptr: run starts
  // (ntiles+1); x_rel: per level-1 block the R+1 row offsets inside its run
  // (stored with a stride of R+1 rounded up to a multiple of 4);
  // lmapx: lower entry -> slot, -1 for same-block entries.
  std::vector<int64_t> fx_ptr, bx_ptr;
  std::vector<int32_t> fx_rel, bx_rel, fx_col, bx_col;
  std::vector<int64_t> lmapx_f, lmapx_b;
  int64_t max_x_f = 0, max_x_b = 0, max_xrow_f = 0, max_xrow_b = 0;

  // Per level-1 block ("unit") records, rec_ints int32 each:
  //   [0] o_len, [1] i_len, [2..3] o_begin, [4..5] i_begin (int64 halves),
  //   [6 .. 6+bs] o_rel, [7+bs .. 7+2bs] i_rel
  // o = the unit's run of other-color (or, for SpMV, all) entries, i = its
  // same-block run; *_rel are the slice starts inside each run.
  int32_t rec_ints = 0;
  std::vector<int32_t> rec_f, rec_b, rec_a;
  int64_t max_o_f = 0, max_i_f = 0, max_o_b = 0, max_i_b = 0, max_a = 0;
};

// Validates the CSR and computes every host-side structure.  Returns
// HBMC_OK or an error with a message in err.
hbmc_status build_host(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                       int32_t bs, int32_t w, const hbmc_options &opt, HostLayout &h,
                       std::string &err);

// Per-unit records of h from its slice pointer arrays (h.rec_*, h.max_*).
hbmc_status make_records(HostLayout &h, std::string &err);

// The variable-slice-height SpMV layout (h.vs_*) from h's SELL layout.
hbmc_status plan_vslice(HostLayout &h, int32_t cost, std::string &err);

// The batched solver's view of its systems (see batch_host.cpp).
struct BatchMeta {
  int32_t nsys = 0, nc = 0;
  std::vector<int64_t> n, n_pad, orig0;   // per system; orig0[s] = first row of system s in
                                          // the concatenated original-order vectors
  std::vector<int32_t> nc_sys;
  std::vector<int32_t> unit_sys;          // global level-1 block -> system
  std::vector<int64_t> cu_start, cu_count;  // [s * nc + c]: system s's blocks of color c
};

hbmc_status build_batch_host(int32_t nsys, const hbmc_system *sys, int32_t bs, int32_t w,
                             const hbmc_options &opt, HostLayout &g, BatchMeta &meta, std::string &err);

// A device context around a prepared host layout, and a read-only view of a
// context for entry points in other translation units.
hbmc_status make_ctx_from_layout(HostLayout &&h, const hbmc_options &opt, hbmc_ctx **out, std::string &err);

// Device scalars of one solve.
struct Scalars {
  double rho, rho_new, beta, pq, alpha, rr, bb, bnorm, relres, tol, true_relres;
  long long iters, maxit;
  double omega, rho_old, rv, tt, ts;  // BiCGStab scalars
  int half;    // BiCGStab: the half step met the tolerance (x += alpha ph still owed)
  int status;  // 0 running, 1 converged, 2 maxit reached, 3 breakdown
  int done;    // nonzero: every further kernel of the solve returns at once
  int zero_x;  // b == 0: the solution is x = 0
  int timeout;  // a bounded device-side wait ran out
  long long bad_row;  // IC(0): smallest failing padded row, or a large sentinel
  unsigned int cnt[8];        // last-block counters of the reductions
  const double *user_b;       // per-call vectors in the original ordering
  double *user_x;
};

enum { ST_RUNNING = 0, ST_CONVERGED = 1, ST_MAXIT = 2, ST_BREAKDOWN = 3 };
enum { CNT_RES = 0, CNT_PQ = 1, CNT_RR = 2, CNT_RZ = 3, CNT_TRUE = 4, CNT_S = 5, CNT_W = 6, CNT_RHO = 7 };

// Shared memory of one warp in the warp-per-unit kernels (byte offsets), and
// warps per CUDA block; wpb = 0 means the plan does not fit.
struct WarpPlan {
  uint32_t off_t = 0, off_d = 0, off_iv = 0, off_im = 0, warp_bytes = 0;
  int wpb = 0;
};

// Shared memory of one warp in the bulk-copy-staged warp-per-unit sweeps
// (byte offsets: mbarrier at 0, record at 16); ok = false when 4 warps do
// not fit.
struct TwPlan {
  uint32_t off_ts = 0, off_tin = 0, off_ds = 0, off_iv = 0, off_im = 0, warp_bytes = 0;
  bool ok = false;
};

// Shared memory of the loader-thread sweeps (sweep_wide.cu), byte offsets;
// ok = false when a level-1 block's runs do not fit.
struct WidePlan {
  uint32_t off_xr = 0, off_ts = 0, off_tin = 0, off_ds = 0, off_rr = 0, off_oc = 0, off_vv = 0, off_gv = 0,
           off_iv = 0, off_im = 0, smem_bytes = 0;
  int32_t chunk = 0;  // other-color entries staged per round (the whole run when it fits)
  bool ok = false;
};

// Shared memory of the dependency-driven sweeps (sweep_dag.cu), byte
// offsets; ok = false when a level-1 block's runs do not fit.  resident:
// CUDA blocks of the launch that fit on one SM (registers and shared memory).
struct DagPlan {
  uint32_t off_xr = 0, off_ts = 0, off_tin = 0, off_ds = 0, off_rr = 0, off_oc = 0, off_vv = 0, off_iv = 0,
           off_im = 0, off_pos = 0, smem_bytes = 0;
  int resident = 0;
  bool ok = false;
};

// Shared memory of the SOR sweep kernel (sor.cu), byte offsets.
struct SorPlan {
  uint32_t off_cb = 0, off_bb = 0, off_dd = 0, off_sv = 0, off_ix = 0, smem_bytes = 0;
  bool ok = false;
};

// Stage ring of the bulk-copy-fed SpMV (spmv_tma.cu); stages = 0: not used.
struct SpmvPlan {
  int64_t nslices = 0, nchunks = 0;
  uint32_t off_val = 0, off_p = 0, stage_bytes = 0;
  int stages = 0, blocks_per_sm = 0;
};

struct DeviceLayout;
bool ctx_view(hbmc_ctx *ctx, const DeviceLayout **d, cudaStream_t *stream, int *device, bool *factored,
              std::string **err);

// Device-side copy of the layouts.
struct DeviceLayout {
  int64_t n = 0, n_pad = 0, nnz_lower = 0;
  int32_t bs = 1, w = 1, nc = 0;
  std::vector<int64_t> tile_ptr;  // host copy, for launch geometry
  int64_t *tile_ptr_dev = nullptr;  // device copy (persistent kernel)
  unsigned *pbar = nullptr;         // persistent kernel's grid barrier: arrivals, generation, error

  // sweep launch geometry: level-1 blocks per CUDA block, and the largest
  // same-block coefficient run of one CUDA block (staged in shared memory
  // when it fits)
  int32_t sweep_tpb = 1;
  int32_t sm_count = 1;  // streaming multiprocessors of the device
  int32_t sweep_kernel = 0;  // hbmc_options.sweep_kernel (2 mapped to 0)
  // warp-per-unit kernels: device records and shared-memory plans
  int32_t rec_ints = 0;
  int32_t *rec_f = nullptr, *rec_b = nullptr, *rec_a = nullptr;
  int64_t max_i_f = 0, max_i_b = 0;
  WarpPlan wp_f64_f, wp_f64_b, wp_f32_f, wp_f32_b, wp_spmv;
  TwPlan tw_f64_f, tw_f64_b, tw_f32_f, tw_f32_b;
  TwPlan tw_fb_f64, tw_fb_f32;  // last color, forward and backward in one pass
  SpmvPlan sp;
  SorPlan sor;
  WidePlan wd_f64_f, wd_f64_b, wd_f32_f, wd_f32_b;  // plain-load staging
  WidePlan wt_f64_f, wt_f64_b, wt_f32_f, wt_f32_b;  // bulk-copy staging (w = 32)
  WidePlan ws_f64_f, ws_f64_b, ws_f32_f, ws_f32_b;  // split over several CUDA blocks per level-1 block
  std::vector<uint8_t> wide_f, wide_b;  // per color: 1 = loader-thread sweep, 2 = its split form
  unsigned *ucnt = nullptr;  // per level-1 block arrival counters of the split form (zero between launches)
  // dependency-driven sweeps: per level-1 block what it waits for
  // (forward, backward), the backward sweep's order, level-1 block -> color
  // and color -> level-1 blocks, the completion flags and counters, the
  // ticket counters and abort words ([0] forward, [1] backward), and the test hook (a level-1 block that never publishes,
  // and the bound of every wait)
  int64_t *dep_ptr_f = nullptr, *dep_ptr_b = nullptr, *dag_color_units = nullptr;
  int32_t *dep_f = nullptr, *dep_b = nullptr, *dag_order_b = nullptr, *dag_unit_color = nullptr;
  unsigned *dag_flag_f = nullptr, *dag_flag_b = nullptr, *dag_abort = nullptr;
  unsigned *dag_color_done = nullptr;  // per color, forward then backward (cleared by each launch's last block)
  uint8_t *dag_counted = nullptr;      // per color, forward then backward: some level-1 block waits on its counter
  unsigned *dag_exit = nullptr;        // finished CUDA blocks of the running launch, forward and backward
  unsigned long long *dag_ticket = nullptr;
  DagPlan dg_f64_f, dg_f64_b, dg_f32_f, dg_f32_b;
  int64_t dag_stall = -1;
  uint64_t dag_wait_ns = 4000000000ull;
  int32_t lw = 0;        // log2(w)
  int64_t max_in_f = 0, max_in_b = 0;
  int32_t in_smem_f = 0, in_smem_b = 0;

  int32_t *inv = nullptr, *pi = nullptr;
  int64_t *a_ptr = nullptr;
  int32_t *a_col = nullptr;
  double *a_val = nullptr;
  // split SpMV layout (split = 1 when built with hbmc_options.sell_split)
  int32_t split = 0;
  int64_t n_virt = 0;  // piece rows, a multiple of w
  int64_t *sh_ptr = nullptr, *sp_ptr = nullptr;
  int32_t *sh_col = nullptr, *sp_col = nullptr;
  double *sh_val = nullptr, *sp_val = nullptr;
  uint32_t *sl_mask = nullptr;
  int32_t *sl_first = nullptr, *cmb_ptr = nullptr, *cmb_slot = nullptr;
  double *tsum = nullptr;  // the pieces' sums, n_virt
  // variable-slice-height SpMV layout (vslice = 1 when built with hbmc_options.sell_vslice)
  int32_t vslice = 0;
  uint8_t *vs_c = nullptr;
  int64_t *vs_first = nullptr, *vs_ptr = nullptr;
  int32_t *vs_col = nullptr;
  double *vs_val = nullptr;
  int64_t *fo_ptr = nullptr, *fi_ptr = nullptr, *bo_ptr = nullptr, *bi_ptr = nullptr;
  int32_t *fo_col = nullptr, *bo_col = nullptr;
  uint8_t *fi_m = nullptr, *bi_m = nullptr;
  double *fo_val = nullptr, *fi_val = nullptr, *bo_val = nullptr, *bi_val = nullptr;
  double *dinv = nullptr;   // forward sweep's diagonal scaling (1 / l_ii; all ones for ILU(0))
  double *dinvb = nullptr;  // backward sweep's (1 / l_ii, the same array, for IC(0); 1 / u_ii for ILU(0))
  float *fo_val32 = nullptr, *fi_val32 = nullptr, *bo_val32 = nullptr, *bi_val32 = nullptr;
  float *dinv32 = nullptr, *dinvb32 = nullptr;
  // ILU(0) (nonsymmetric contexts): transposed values, upper rows, the U factor
  int32_t nonsym = 0;
  double *uaval = nullptr, *uval = nullptr, *udiag = nullptr;
  int64_t *urp = nullptr, *upos = nullptr;
  int32_t *uci = nullptr;
  // BiCGStab vectors (nonsymmetric contexts; n_pad + kGuard each)
  double *rh = nullptr, *sv = nullptr, *ph = nullptr;
  int64_t *lrp = nullptr;
  int32_t *lci = nullptr;
  double *laval = nullptr, *adiag = nullptr, *lval = nullptr, *ldiag = nullptr;
  int64_t *lmap_f = nullptr, *lmap_b = nullptr;
  // unpadded other-color runs of the loader-thread sweeps (HostLayout fx_*, bx_*)
  int64_t *fx_ptr = nullptr, *bx_ptr = nullptr, *lmapx_f = nullptr, *lmapx_b = nullptr;
  int32_t *fx_rel = nullptr, *bx_rel = nullptr, *fx_col = nullptr, *bx_col = nullptr;
  double *fx_val = nullptr, *bx_val = nullptr;
  float *fx_val32 = nullptr, *bx_val32 = nullptr;
  // vectors in HBMC order, n_pad + kGuard doubles (guard entries stay 0)
  double *b = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr,
         *y = nullptr, *t = nullptr;
  float *y32 = nullptr, *z32 = nullptr;
  double *part = nullptr;  // reduction partials
  int64_t part_len = 0;
  double *hist = nullptr;
  Scalars *sc = nullptr;
  size_t bytes = 0;
};

// Features of a device layout seen as nsys systems (unit ranges per system and
// color on the device; nullptr: one system spanning the whole layout).
hbmc_status features_on_device(const DeviceLayout &d, int32_t nsys, const int64_t *cu_start_dev,
                               const int64_t *cu_count_dev, const int32_t *nc_sys_dev, float *feat_dev,
                               cudaStream_t s, std::string &err);

}  // namespace hbmc

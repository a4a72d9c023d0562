// Internal declarations shared by the host build, the kernels and the C ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

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

  // SpMV: SELL with slice height w, column-major inside a slice
  std::vector<int64_t> a_ptr;  // nslices+1, entry offsets
  std::vector<int32_t> a_col;
  std::vector<double> a_val;

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
};

// Validates the CSR and computes every host-side structure.  Returns
// HBMC_OK or an error with a message in err.
hbmc_status build_host(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                       int32_t bs, int32_t w, const hbmc_options &opt, HostLayout &h,
                       std::string &err);

// Device scalars of one solve.
struct Scalars {
  double rho, rho_new, beta, pq, alpha, rr, bb, bnorm, relres, tol, true_relres;
  long long iters, maxit;
  int status;  // 0 running, 1 converged, 2 maxit reached, 3 breakdown
  int done;    // nonzero: every further kernel of the solve returns at once
  int zero_x;  // b == 0: the solution is x = 0
  int pad0;
  long long bad_row;  // IC(0): smallest failing padded row, or a large sentinel
  unsigned int cnt[8];        // last-block counters of the reductions
  const double *user_b;       // per-call vectors in the original ordering
  double *user_x;
};

enum { ST_RUNNING = 0, ST_CONVERGED = 1, ST_MAXIT = 2, ST_BREAKDOWN = 3 };
enum { CNT_RES = 0, CNT_PQ = 1, CNT_RR = 2, CNT_RZ = 3, CNT_TRUE = 4 };

// Device-side copy of the layouts.
struct DeviceLayout {
  int64_t n = 0, n_pad = 0, nnz_lower = 0;
  int32_t bs = 1, w = 1, nc = 0;
  std::vector<int64_t> tile_ptr;  // host copy, for launch geometry

  int32_t *inv = nullptr, *pi = nullptr;
  int64_t *a_ptr = nullptr;
  int32_t *a_col = nullptr;
  double *a_val = nullptr;
  int64_t *fo_ptr = nullptr, *fi_ptr = nullptr, *bo_ptr = nullptr, *bi_ptr = nullptr;
  int32_t *fo_col = nullptr, *bo_col = nullptr;
  uint8_t *fi_m = nullptr, *bi_m = nullptr;
  double *fo_val = nullptr, *fi_val = nullptr, *bo_val = nullptr, *bi_val = nullptr;
  double *dinv = nullptr;
  float *fo_val32 = nullptr, *fi_val32 = nullptr, *bo_val32 = nullptr, *bi_val32 = nullptr;
  float *dinv32 = nullptr;
  int64_t *lrp = nullptr;
  int32_t *lci = nullptr;
  double *laval = nullptr, *adiag = nullptr, *lval = nullptr, *ldiag = nullptr;
  int64_t *lmap_f = nullptr, *lmap_b = nullptr;
  // vectors in HBMC order, n_pad + kGuard doubles (guard entries stay 0)
  double *b = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr,
         *y = nullptr, *t = nullptr;
  float *y32 = nullptr;
  double *part = nullptr;  // reduction partials
  int64_t part_len = 0;
  double *hist = nullptr;
  Scalars *sc = nullptr;
  size_t bytes = 0;
};

}  // namespace hbmc

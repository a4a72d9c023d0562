// CUDA kernels of the HBMC-ICCG solve (sm_103a) and the sequences that
// enqueue them.
//
// Substitutions (Section 4.2.2): a color is one launch (the n_c - 1 thread
// synchronizations of Section 4.3.3 become kernel boundaries); its level-1
// blocks are independent (Eq. "BAMC3") and each CUDA block takes whole
// level-1 blocks.  Inside one, lane j owns BMC block j and the bs steps of
// Eqs. "y2-2"/"y2-3" run in order, each step touching w consecutive rows, so
// every slice column of the SELL layout is one coalesced load.  The
// couplings to other colors (Eq. "for3") do not depend on the step chain and
// are computed first with one thread per row; the chain itself only involves
// the lane's own earlier steps and runs out of shared memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>

#include "hbmc_internal.h"
#include "device_util.cuh"
#include "kernels.h"

namespace hbmc {
namespace {

constexpr int kRowThreads = 256;
constexpr int kSweepThreads = 128;

// ---------------------------------------------------------------------------
// Permutations (Section 3, Eq. "xbar": xbar = P x)
// ---------------------------------------------------------------------------

// dst[k] = src[inv[k]] (0 for dummies); which = 0/1: take src from the solve's
// user b / x pointers in the scalars block instead.
__global__ void k_gather_in(const double *src, double *dst, const int32_t *__restrict__ inv,
                            int64_t n_pad, const Scalars *sc, int which) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_pad) return;
  if (which == 0) src = sc->user_b;
  if (which == 1) src = sc->user_x;
  const int32_t i = inv[k];
  dst[k] = i >= 0 ? src[i] : 0.0;
}

// dst[i] = src[pi[i]]; with sc given, dst is the solve's user x and a zero
// right-hand side gives x = 0.
__global__ void k_gather_out(const double *src, double *dst, const int32_t *__restrict__ pi,
                             int64_t n, const Scalars *sc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (sc) {
    sc->user_x[i] = sc->zero_x ? 0.0 : src[pi[i]];
  } else {
    dst[i] = src[pi[i]];
  }
}

__global__ void k_widen(const float *src, double *dst, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (double)src[i];
}

__global__ void k_narrow(const double *src, float *dst, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (float)src[i];
}

// ---------------------------------------------------------------------------
// SpMV with SELL slices of w rows (Section 4.3.2); terms in ascending column
// order, accumulated from zero with fused multiply-adds.
// ---------------------------------------------------------------------------

__device__ __forceinline__ double sell_row(const int64_t *__restrict__ a_ptr,
                                           const int32_t *__restrict__ a_col,
                                           const double *__restrict__ a_val, int w, int lw,
                                           int64_t row, const double *x) {
  const int64_t s = row >> lw;
  const int j = (int)(row & (w - 1));
  const int64_t pe = a_ptr[s + 1];
  double acc = 0.0;
  for (int64_t p = a_ptr[s] + j; p < pe; p += w) acc = fma(a_val[p], __ldg(x + a_col[p]), acc);
  return acc;
}



// mode 0: initial residual r = b - A x with ||b||^2 and ||r||^2;
// mode 1: true residual after the solve, ||b - A x||^2 only (t is scratch).
template <int kMode>
__global__ void __launch_bounds__(kRowThreads)
    k_residual(const int64_t *__restrict__ a_ptr, const int32_t *__restrict__ a_col,
               const double *__restrict__ a_val, int w, int lw, int64_t n_pad, const double *b,
               const double *x, double *r, double *part, Scalars *sc, double *hist) {
  double bb = 0.0, rr = 0.0;
  FOR_ROWS(row, n_pad) {
    const double acc = sell_row(a_ptr, a_col, a_val, w, lw, row, x);
    const double bi = b[row];
    const double ri = bi - acc;
    if (kMode == 0) r[row] = ri;
    bb = fma(bi, bi, bb);
    rr = fma(ri, ri, rr);
  }
  double v[2];
  v[0] = block_sum<kRowThreads>(bb);
  v[1] = block_sum<kRowThreads>(rr);
  const int cid = kMode == 0 ? CNT_RES : CNT_TRUE;
  if (!publish(part + 2 * blockIdx.x, v, 2, &sc->cnt[cid], gridDim.x)) return;
  const double sbb = gather_partials<kRowThreads>(part, gridDim.x, 2, 0);
  const double srr = gather_partials<kRowThreads>(part, gridDim.x, 2, 1);
  if (threadIdx.x != 0) return;
  sc->cnt[cid] = 0;
  if (kMode == 1) {
    sc->true_relres = sc->bnorm > 0.0 ? sqrt(srr) / sc->bnorm : 0.0;
    return;
  }
  sc->bb = sbb;
  sc->bnorm = sqrt(sbb);
  sc->iters = 0;
  if (sc->bnorm == 0.0) {
    sc->zero_x = 1;
    sc->relres = 0.0;
    hist[0] = 0.0;
    sc->status = ST_CONVERGED;
    sc->done = 1;
    return;
  }
  const double res = sqrt(srr) / sc->bnorm;
  sc->relres = res;
  hist[0] = res;
  if (res < sc->tol) {
    sc->status = ST_CONVERGED;
    sc->done = 1;
  } else if (sc->maxit <= 0) {
    sc->status = ST_MAXIT;
    sc->done = 1;
  }
}

// q = A p, with p.q and alpha = rho / p.q.
template <bool kDot>
__global__ void __launch_bounds__(kRowThreads)
    k_spmv(const int64_t *__restrict__ a_ptr, const int32_t *__restrict__ a_col,
           const double *__restrict__ a_val, int w, int lw, int64_t n_pad, const double *p,
           double *q, double *part, Scalars *sc) {
  if (kDot && sc->done) return;
  double pq = 0.0;
  FOR_ROWS(row, n_pad) {
    const double acc = sell_row(a_ptr, a_col, a_val, w, lw, row, p);
    q[row] = acc;
    if (kDot) pq = fma(p[row], acc, pq);
  }
  if (!kDot) return;
  double v = block_sum<kRowThreads>(pq);
  if (!publish(part + blockIdx.x, &v, 1, &sc->cnt[CNT_PQ], gridDim.x)) return;
  const double s = gather_partials<kRowThreads>(part, gridDim.x, 1, 0);
  if (threadIdx.x != 0) return;
  sc->cnt[CNT_PQ] = 0;
  sc->pq = s;
  if (!(s > 0.0) || !finite(s)) {
    sc->status = ST_BREAKDOWN;
    sc->done = 1;
    return;
  }
  sc->alpha = sc->rho / s;
}

// Variable-slice-height SpMV (hbmc_options.sell_vslice): row j of slice s
// lies in sub-slice vs_first[s] + j / C (C = vs_c[s]) at position j % C,
// its entry t at vs_ptr[sub] + t * C + position.  The row's terms are summed
// from zero in ascending column order, as in the plain layout, so the
// product is the same bits; only the padding differs.
template <bool kDot>
__global__ void __launch_bounds__(kRowThreads)
    k_spmv_vs(const uint8_t *__restrict__ vs_c, const int64_t *__restrict__ vs_first,
              const int64_t *__restrict__ vs_ptr, const int32_t *__restrict__ col, const double *__restrict__ val,
              int w, int lw, int64_t n_pad, const double *p, double *q, double *part, Scalars *sc) {
  if (kDot && sc->done) return;
  double pq = 0.0;
  FOR_ROWS(row, n_pad) {
    const double acc = vs_row(vs_c, vs_first, vs_ptr, col, val, w, lw, row, p);
    q[row] = acc;
    if (kDot) pq = fma(p[row], acc, pq);
  }
  if (!kDot) return;
  double v = block_sum<kRowThreads>(pq);
  if (!publish(part + blockIdx.x, &v, 1, &sc->cnt[CNT_PQ], gridDim.x)) return;
  const double t = gather_partials<kRowThreads>(part, gridDim.x, 1, 0);
  if (threadIdx.x != 0) return;
  sc->cnt[CNT_PQ] = 0;
  sc->pq = t;
  if (!(t > 0.0) || !finite(t)) {
    sc->status = ST_BREAKDOWN;
    sc->done = 1;
    return;
  }
  sc->alpha = sc->rho / t;
}

// Row-split SpMV (Section 5.2.2's remedy for slices whose rows differ much
// in length).  First the pieces: every cut-off piece is a row of its own in
// a SELL layout of slices of w pieces, summed from zero in ascending column
// order.
__global__ void __launch_bounds__(kRowThreads)
    k_spmv_pieces(const int64_t *__restrict__ sp_ptr, const int32_t *__restrict__ sp_col,
                  const double *__restrict__ sp_val, int w, int lw, int64_t n_virt, const double *p,
                  double *tsum, const Scalars *sc) {
  if (sc && sc->done) return;  // sc is given inside the CG loop only
  FOR_ROWS(v, n_virt) tsum[v] = sell_row(sp_ptr, sp_col, sp_val, w, lw, v, p);
}

struct SplitArgs {
  const int64_t *sh_ptr;
  const int32_t *sh_col;
  const double *sh_val;
  const uint32_t *sl_mask;
  const int32_t *sl_first, *cmb_ptr, *cmb_slot;
  const double *tsum;
};

// Then every row: its head (the slice's first t entries, from zero, ascending
// columns) plus, for a split row, its pieces' sums added in piece order --
// the oracle's q_i = ((S_0 + S_1) + S_2) + ... -- with p.q and alpha as in
// k_spmv.
template <bool kDot>
__global__ void __launch_bounds__(kRowThreads)
    k_spmv_split(const SplitArgs a, int w, int lw, int64_t n_pad, const double *p, double *q, double *part,
                 Scalars *sc) {
  if (kDot && sc->done) return;
  double pq = 0.0;
  FOR_ROWS(row, n_pad) {
    double acc = sell_row(a.sh_ptr, a.sh_col, a.sh_val, w, lw, row, p);
    const int64_t s = row >> lw;
    const int j = (int)(row & (w - 1));
    const uint32_t mk = a.sl_mask[s];
    if ((mk >> j) & 1u) {
      const int k = a.sl_first[s] + __popc(mk & ((1u << j) - 1u));
      for (int c = a.cmb_ptr[k]; c < a.cmb_ptr[k + 1]; ++c) acc = __dadd_rn(acc, a.tsum[a.cmb_slot[c]]);
    }
    q[row] = acc;
    if (kDot) pq = fma(p[row], acc, pq);
  }
  if (!kDot) return;
  double v = block_sum<kRowThreads>(pq);
  if (!publish(part + blockIdx.x, &v, 1, &sc->cnt[CNT_PQ], gridDim.x)) return;
  const double sum = gather_partials<kRowThreads>(part, gridDim.x, 1, 0);
  if (threadIdx.x != 0) return;
  sc->cnt[CNT_PQ] = 0;
  sc->pq = sum;
  if (!(sum > 0.0) || !finite(sum)) {
    sc->status = ST_BREAKDOWN;
    sc->done = 1;
    return;
  }
  sc->alpha = sc->rho / sum;
}

// x += alpha p, r -= alpha q, ||r||^2, iteration count and stopping test.
__global__ void __launch_bounds__(kRowThreads)
    k_update_xr(int64_t n_pad, const double *p, const double *q, double *x, double *r,
                double *part, Scalars *sc, double *hist, int use_cond,
                cudaGraphConditionalHandle handle) {
  if (sc->done) {
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(handle, 0);
    return;
  }
  const double alpha = sc->alpha;
  double rr = 0.0;
  FOR_ROWS(row, n_pad) {
    x[row] = fma(alpha, p[row], x[row]);
    const double ri = fma(-alpha, q[row], r[row]);
    r[row] = ri;
    rr = fma(ri, ri, rr);
  }
  double v = block_sum<kRowThreads>(rr);
  if (!publish(part + blockIdx.x, &v, 1, &sc->cnt[CNT_RR], gridDim.x)) return;
  const double s = gather_partials<kRowThreads>(part, gridDim.x, 1, 0);
  if (threadIdx.x != 0) return;
  sc->cnt[CNT_RR] = 0;
  sc->rr = s;
  const long long k = sc->iters + 1;
  sc->iters = k;
  const double res = sqrt(s) / sc->bnorm;
  sc->relres = res;
  if (k < kHistCap) hist[k] = res;
  if (res < sc->tol) {
    sc->status = ST_CONVERGED;
    sc->done = 1;
  } else if (k >= sc->maxit) {
    sc->status = ST_MAXIT;
    sc->done = 1;
  }
  if (sc->done && use_cond) cudaGraphSetConditional(handle, 0);
}

// p = z + beta p (mode 1), or p = z at the start (mode 0).
__global__ void __launch_bounds__(kRowThreads)
    k_update_p(int64_t n_pad, const double *z, double *p, Scalars *sc, int mode, int use_cond,
               cudaGraphConditionalHandle handle) {
  if (sc->done) {
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(handle, 0);
    return;
  }
  if (mode == 0) {
    FOR_ROWS(row, n_pad) p[row] = z[row];
  } else {
    const double beta = sc->beta;
    FOR_ROWS(row, n_pad) p[row] = fma(beta, p[row], z[row]);
  }
}

// ---------------------------------------------------------------------------
// Substitutions, one color per launch.  A CUDA block holds tpb whole level-1
// blocks (tpb * bs * w rows).  Forward, color c (Eqs. "for2", "for3"):
//   phase 1, one thread per row:  t_i = r_i - sum_{j in earlier colors} l_ij y_j
//            (q_c of Eq. "for3"; these gathers do not depend on the step chain)
//   phase 2, lane j of each level-1 block, steps l = 1..bs (Eqs. "y2-2", "y2-3"):
//            y_i = (t_i - sum_{m<l} l_{i,(m,j)} y_(m,j)) * dinv_i, all in shared memory
//   phase 3, one thread per row: store y.
// Backward, color c, colors n_c..1 and steps bs..1, with U = L^T.
// The per-row term order (other colors first, then the same BMC block, each
// farthest from the diagonal first) matches the oracle exactly.
// ---------------------------------------------------------------------------
constexpr int kTileThreads = 256;

template <typename T>
struct SweepArgs {
  const int64_t *o_ptr, *i_ptr;
  const int32_t *o_col;
  const uint8_t *i_m;
  const T *o_val, *i_val, *dinv;
  int bs, w, lw, tpb, in_smem;
  int64_t max_in, tile0, ntiles;
};

template <typename T>
struct SweepSmem {
  T *tv, *dv, *iv;
  int32_t *ip;
  uint8_t *im;
};

template <typename T>
__device__ __forceinline__ SweepSmem<T> carve(unsigned char *raw, const SweepArgs<T> &a) {
  SweepSmem<T> m;
  const int cap = a.tpb * (a.bs << a.lw);
  m.tv = reinterpret_cast<T *>(raw);
  m.dv = m.tv + cap;
  m.ip = reinterpret_cast<int32_t *>(m.dv + cap);
  uintptr_t q = reinterpret_cast<uintptr_t>(m.ip + a.tpb * a.bs + 1);
  q = (q + 15) & ~uintptr_t(15);
  m.iv = reinterpret_cast<T *>(q);
  m.im = reinterpret_cast<uint8_t *>(m.iv + (a.in_smem ? a.max_in : 0));
  return m;
}

// Shared prologue: slice offsets of the same-block runs and, when they fit,
// the runs themselves.  Returns the global offset of the block's first run.
template <typename T>
__device__ __forceinline__ int64_t stage_runs(const SweepArgs<T> &a, const SweepSmem<T> &m,
                                              int64_t s_begin, int nsl) {
  const int64_t ib0 = a.i_ptr[s_begin];
  for (int k = threadIdx.x; k <= nsl; k += kTileThreads) m.ip[k] = (int32_t)(a.i_ptr[s_begin + k] - ib0);
  if (a.in_smem) {
    const int64_t cnt = a.i_ptr[s_begin + nsl] - ib0;
    for (int64_t e = threadIdx.x; e < cnt; e += kTileThreads) {
      m.iv[e] = a.i_val[ib0 + e];
      m.im[e] = a.i_m[ib0 + e];
    }
  }
  return ib0;
}

template <typename T, typename Y>
__global__ void __launch_bounds__(kTileThreads)
    k_fwd(const SweepArgs<T> a, const double *__restrict__ r, Y *y, const Scalars *sc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (sc && sc->done) return;
  const SweepSmem<T> m = carve(smem_raw, a);
  const int R = a.bs << a.lw;
  const int64_t bt0 = a.tile0 + (int64_t)blockIdx.x * a.tpb;
  const int ntl = (int)min((int64_t)a.tpb, a.tile0 + a.ntiles - bt0);
  const int nrows = ntl * R;
  const int64_t row0 = bt0 * R;
  const int64_t ib0 = stage_runs(a, m, bt0 * a.bs, ntl * a.bs);
#pragma unroll 4
  for (int lr = threadIdx.x; lr < nrows; lr += kTileThreads) {
    const int64_t row = row0 + lr;
    const int64_t s = row >> a.lw;
    const int j = (int)(row & (a.w - 1));
    T acc = (T)r[row];
    const int64_t pe = a.o_ptr[s + 1];
    for (int64_t p = a.o_ptr[s] + j; p < pe; p += a.w) acc = fma(-a.o_val[p], (T)y[a.o_col[p]], acc);
    m.tv[lr] = acc;
    m.dv[lr] = a.dinv[row];
  }
  __syncthreads();
  if (threadIdx.x < ntl * a.w) {
    const int tl = threadIdx.x >> a.lw, j = threadIdx.x & (a.w - 1);
    T *tt = m.tv + tl * R;
    const T *dd = m.dv + tl * R;
    for (int l = 0; l < a.bs; ++l) {
      const int k = tl * a.bs + l;
      T acc = tt[(l << a.lw) + j];
      const int pe = m.ip[k + 1];
      for (int p = m.ip[k] + j; p < pe; p += a.w) {
        const int mm = a.in_smem ? m.im[p] : a.i_m[ib0 + p];
        const T v = a.in_smem ? m.iv[p] : a.i_val[ib0 + p];
        acc = fma(-v, tt[(mm << a.lw) + j], acc);
      }
      tt[(l << a.lw) + j] = acc * dd[(l << a.lw) + j];
    }
  }
  __syncthreads();
#pragma unroll 4
  for (int lr = threadIdx.x; lr < nrows; lr += kTileThreads) y[row0 + lr] = (Y)m.tv[lr];
}

// dot_mode 1: initial rho = r.z; 2: rho and beta = rho_new / rho.  The launch
// of the last color (color 1) finishes the sum over every color's partials.
template <typename T, typename Y>
__global__ void __launch_bounds__(kTileThreads)
    k_bwd(const SweepArgs<T> a, const Y *__restrict__ yin, double *z, float *z32, const double *__restrict__ r,
          Scalars *sc, int dot_mode, double *part, int64_t part_off, int last_launch,
          int64_t part_total) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (sc && sc->done) return;
  const SweepSmem<T> m = carve(smem_raw, a);
  const int R = a.bs << a.lw;
  const int64_t bt0 = a.tile0 + (int64_t)blockIdx.x * a.tpb;
  const int ntl = (int)min((int64_t)a.tpb, a.tile0 + a.ntiles - bt0);
  const int nrows = ntl * R;
  const int64_t row0 = bt0 * R;
  const int64_t ib0 = stage_runs(a, m, bt0 * a.bs, ntl * a.bs);
#pragma unroll 4
  for (int lr = threadIdx.x; lr < nrows; lr += kTileThreads) {
    const int64_t row = row0 + lr;
    const int64_t s = row >> a.lw;
    const int j = (int)(row & (a.w - 1));
    T acc = (T)yin[row];
    const int64_t pe = a.o_ptr[s + 1];
    const T *zg = zgather<T>(z, z32);
    for (int64_t p = a.o_ptr[s] + j; p < pe; p += a.w) acc = fma(-a.o_val[p], zg[a.o_col[p]], acc);
    m.tv[lr] = acc;
    m.dv[lr] = a.dinv[row];
  }
  __syncthreads();
  if (threadIdx.x < ntl * a.w) {
    const int tl = threadIdx.x >> a.lw, j = threadIdx.x & (a.w - 1);
    T *tt = m.tv + tl * R;
    const T *dd = m.dv + tl * R;
    for (int l = a.bs - 1; l >= 0; --l) {
      const int k = tl * a.bs + l;
      T acc = tt[(l << a.lw) + j];
      const int pe = m.ip[k + 1];
      for (int p = m.ip[k] + j; p < pe; p += a.w) {
        const int mm = a.in_smem ? m.im[p] : a.i_m[ib0 + p];
        const T v = a.in_smem ? m.iv[p] : a.i_val[ib0 + p];
        acc = fma(-v, tt[(mm << a.lw) + j], acc);
      }
      tt[(l << a.lw) + j] = acc * dd[(l << a.lw) + j];
    }
  }
  __syncthreads();
  double rz = 0.0;
  for (int lr = threadIdx.x; lr < nrows; lr += kTileThreads) {
    const double zv = (double)m.tv[lr];
    z[row0 + lr] = zv;
    if constexpr (sizeof(T) == 4) z32[row0 + lr] = m.tv[lr];
    if (dot_mode) rz = fma(r[row0 + lr], zv, rz);
  }
  if (!dot_mode) return;
  const double v = block_sum<kTileThreads>(rz);
  if (threadIdx.x == 0) part[part_off + blockIdx.x] = v;
  if (!last_launch) return;
  __shared__ unsigned s_last;
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(&sc->cnt[CNT_RZ], 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  const double rho_new = gather_partials<kTileThreads>(part, part_total, 1, 0);
  if (threadIdx.x != 0) return;
  sc->cnt[CNT_RZ] = 0;
  sc->rho_new = rho_new;
  if (!(rho_new > 0.0) || !finite(rho_new)) {
    sc->status = ST_BREAKDOWN;
    sc->done = 1;
    return;
  }
  if (dot_mode == 2) sc->beta = rho_new / sc->rho;
  sc->rho = rho_new;
}

// ---------------------------------------------------------------------------
// IC(0), one color (Section 2, Eq. "ILU"; shifted diagonal of Section 5.1).
// Row i of a color depends on rows of earlier colors and on earlier steps of
// its own BMC block only, so the level-1 / lane / step mapping of the
// substitutions applies unchanged.
//   l_ij = (a_ij - sum_k l_ik l_jk) / l_jj  (k ascending, k in both patterns)
//   l_ii = sqrt((1 + shift) a_ii - sum_k l_ik^2)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSweepThreads)
    k_ic0(const int64_t *__restrict__ lrp, const int32_t *__restrict__ lci,
          const double *__restrict__ laval, const double *__restrict__ adiag, double scale,
          double *lval, double *ldiag, double *dinv, int bs, int w, int64_t tile0, int64_t ntiles,
          Scalars *sc) {
  if (sc->bad_row != LLONG_MAX) return;  // an earlier color failed
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tl = g / w;
  if (tl >= ntiles) return;
  const int j = (int)(g - tl * w);
  const int64_t s0 = (tile0 + tl) * bs;
  for (int l = 0; l < bs; ++l) {
    const int64_t i = (s0 + l) * w + j;
    const int64_t e0 = lrp[i], e1 = lrp[i + 1];
    for (int64_t e = e0; e < e1; ++e) {
      const int64_t jj = lci[e];
      double s = laval[e];
      int64_t p = e0, q = lrp[jj];
      const int64_t qe = lrp[jj + 1];
      while (p < e && q < qe) {
        const int32_t cp = lci[p], cq = lci[q];
        if (cp == cq) {
          s = fma(-lval[p], lval[q], s);
          ++p;
          ++q;
        } else if (cp < cq) {
          ++p;
        } else {
          ++q;
        }
      }
      lval[e] = s / ldiag[jj];
    }
    double d = scale * adiag[i];
    for (int64_t e = e0; e < e1; ++e) d = fma(-lval[e], lval[e], d);
    if (!(d > 0.0) || !finite(d)) {
      atomicMin(&sc->bad_row, (long long)i);
      ldiag[i] = nan("");
      dinv[i] = nan("");
      continue;
    }
    const double ld = sqrt(d);
    ldiag[i] = ld;
    dinv[i] = 1.0 / ld;
  }
}

// Spread the factor into the substitution layouts (and their FP32 copies).
// lval feeds the forward layout, bval the backward one (the same array for
// IC(0), whose U is L^T; U's values for ILU(0)).
struct ScatterArgs {
  const int64_t *lmap_f, *lmap_b, *lmapx_f, *lmapx_b;
  double *fo, *fi, *bo, *bi, *fx, *bx;
  float *fo32, *fi32, *bo32, *bi32, *fx32, *bx32;  // null: no FP32 copies
};

__global__ void k_scatter_factor(int64_t nnz_lower, const double *__restrict__ lval,
                                 const double *__restrict__ bval, const ScatterArgs a) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz_lower) return;
  const double v = lval[e], u = bval[e];
  const int64_t f = a.lmap_f[e], b = a.lmap_b[e];
  const int64_t xf = a.lmapx_f ? a.lmapx_f[e] : -1, xb = a.lmapx_b ? a.lmapx_b[e] : -1;
  if (f >= 0) a.fo[f] = v; else a.fi[-f - 1] = v;
  if (b >= 0) a.bo[b] = u; else a.bi[-b - 1] = u;
  if (xf >= 0) a.fx[xf] = v;
  if (xb >= 0) a.bx[xb] = u;
  if (a.fo32) {
    if (f >= 0) a.fo32[f] = (float)v; else a.fi32[-f - 1] = (float)v;
    if (b >= 0) a.bo32[b] = (float)u; else a.bi32[-b - 1] = (float)u;
    if (xf >= 0) a.fx32[xf] = (float)v;
    if (xb >= 0) a.bx32[xb] = (float)u;
  }
}

__global__ void k_set_bad_row(Scalars *sc) {
  sc->bad_row = LLONG_MAX;
  sc->done = 0;
}

inline unsigned blocks_for(int64_t n, int nt) { return (unsigned)((n + nt - 1) / nt); }

// Grid of the row kernels: enough CUDA blocks to fill every SM a few times
// over, never more than one row per thread.
constexpr int kRowBlocksPerSm = 8;
inline unsigned row_grid(const DeviceLayout &d) {
  const unsigned full = blocks_for(d.n_pad, kRowThreads);
  const unsigned cap = (unsigned)(d.sm_count * kRowBlocksPerSm);
  return full < cap ? full : cap;
}

}  // namespace

// ---------------------------------------------------------------------------
// Enqueue sequences
// ---------------------------------------------------------------------------

constexpr int kSweepSmemCap = 200 * 1024;
constexpr int64_t kRunSmemBytes = 64 * 1024;

cudaError_t setup_kernels() {
  cudaError_t e = cudaSuccess;
  if ((e = cudaFuncSetAttribute(k_fwd<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSweepSmemCap))) return e;
  if ((e = cudaFuncSetAttribute(k_bwd<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSweepSmemCap))) return e;
  if ((e = cudaFuncSetAttribute(k_fwd<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSweepSmemCap))) return e;
  if ((e = cudaFuncSetAttribute(k_bwd<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSweepSmemCap))) return e;
  return e;
}

// Level-1 blocks per CUDA block of the sweeps, and the longest same-block
// run a CUDA block stages (forward and backward layouts).
void sweep_geometry(const HostLayout &h, DeviceLayout &d, int tpb) {
  const int R = h.bs * h.w;
  d.sweep_tpb = tpb > 0 ? tpb : (R >= kTileThreads ? 1 : kTileThreads / R);
  d.max_in_f = d.max_in_b = 0;
  for (int c = 0; c < h.nc; ++c)
    for (int64_t t = h.tile_ptr[c]; t < h.tile_ptr[c + 1]; t += d.sweep_tpb) {
      const int64_t te = std::min<int64_t>(t + d.sweep_tpb, h.tile_ptr[c + 1]);
      d.max_in_f = std::max(d.max_in_f, h.fi_ptr[te * h.bs] - h.fi_ptr[t * h.bs]);
      d.max_in_b = std::max(d.max_in_b, h.bi_ptr[te * h.bs] - h.bi_ptr[t * h.bs]);
    }
}

int64_t partials_needed(const DeviceLayout &d) {
  int64_t sweep = 0;
  for (int c = 0; c < d.nc; ++c) sweep += (d.tile_ptr[c + 1] - d.tile_ptr[c] + d.sweep_tpb - 1) / d.sweep_tpb;
  const int64_t rows = 2 * (int64_t)row_grid(d);
  return std::max(std::max(sweep, rows), std::max(std::max(warp_partials_needed(d), tw_partials_needed(d)), std::max(spmv_tma_partials_needed(d), d.nc > 0 ? d.tile_ptr[d.nc] : (int64_t)0))) + 64;
}

namespace {

template <typename T>
SweepArgs<T> sweep_args(const DeviceLayout &d, bool fwd, int c) {
  SweepArgs<T> a;
  a.o_ptr = fwd ? d.fo_ptr : d.bo_ptr;
  a.i_ptr = fwd ? d.fi_ptr : d.bi_ptr;
  a.o_col = fwd ? d.fo_col : d.bo_col;
  a.i_m = fwd ? d.fi_m : d.bi_m;
  if constexpr (sizeof(T) == 8) {
    a.o_val = (const T *)(fwd ? d.fo_val : d.bo_val);
    a.i_val = (const T *)(fwd ? d.fi_val : d.bi_val);
    a.dinv = (const T *)(fwd ? d.dinv : d.dinvb);
  } else {
    a.o_val = (const T *)(fwd ? d.fo_val32 : d.bo_val32);
    a.i_val = (const T *)(fwd ? d.fi_val32 : d.bi_val32);
    a.dinv = (const T *)(fwd ? d.dinv32 : d.dinvb32);
  }
  a.bs = d.bs;
  a.w = d.w;
  a.lw = 0;
  while ((1 << a.lw) < d.w) ++a.lw;
  a.tpb = d.sweep_tpb;
  a.max_in = fwd ? d.max_in_f : d.max_in_b;
  a.in_smem = a.max_in * (int64_t)(sizeof(T) + 1) <= kRunSmemBytes ? 1 : 0;
  a.tile0 = d.tile_ptr[c];
  a.ntiles = d.tile_ptr[c + 1] - d.tile_ptr[c];
  return a;
}

template <typename T>
size_t sweep_smem(const SweepArgs<T> &a) {
  const size_t cap = (size_t)a.tpb * (a.bs << a.lw);
  size_t b = 2 * cap * sizeof(T) + (size_t)(a.tpb * a.bs + 1) * sizeof(int32_t);
  b = (b + 15) & ~size_t(15);
  if (a.in_smem) b += (size_t)a.max_in * (sizeof(T) + 1);
  return b;
}

unsigned sweep_grid(const DeviceLayout &d, int c) {
  return (unsigned)((d.tile_ptr[c + 1] - d.tile_ptr[c] + d.sweep_tpb - 1) / d.sweep_tpb);
}

}  // namespace

void enqueue_gather_in(const DeviceLayout &d, const double *src, double *dst, int which, cudaStream_t s) {
  k_gather_in<<<blocks_for(d.n_pad, kRowThreads), kRowThreads, 0, s>>>(src, dst, d.inv, d.n_pad, d.sc, which);
}

void enqueue_gather_out(const DeviceLayout &d, const double *src, double *dst, bool to_user, cudaStream_t s) {
  k_gather_out<<<blocks_for(d.n, kRowThreads), kRowThreads, 0, s>>>(src, dst, d.pi, d.n, to_user ? d.sc : nullptr);
}

void enqueue_widen(const float *src, double *dst, int64_t n, cudaStream_t s) {
  k_widen<<<blocks_for(n, kRowThreads), kRowThreads, 0, s>>>(src, dst, n);
}

// The integer-operation conversions of the FP32 substitutions on given
// values (test hook: they must equal the casts bit for bit).
__global__ void k_convert_ieee(const double *din, float *fout, const float *fin, double *dout, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    fout[i] = narrow_f64(din[i]);
    dout[i] = widen_f32(fin[i]);
  }
}

void enqueue_convert_ieee(const double *din, float *fout, const float *fin, double *dout, int64_t n,
                          cudaStream_t s) {
  if (n > 0) k_convert_ieee<<<blocks_for(n, kRowThreads), kRowThreads, 0, s>>>(din, fout, fin, dout, n);
}

void enqueue_narrow(const double *src, float *dst, int64_t n, cudaStream_t s) {
  k_narrow<<<blocks_for(n, kRowThreads), kRowThreads, 0, s>>>(src, dst, n);
}

void enqueue_spmv(const DeviceLayout &d, const double *p, double *q, bool dot, cudaStream_t s) {
  if (d.split) {
    if (d.n_virt > 0) {
      const unsigned g = (unsigned)std::min<int64_t>(row_grid(d), blocks_for(d.n_virt, kRowThreads));
      k_spmv_pieces<<<g, kRowThreads, 0, s>>>(d.sp_ptr, d.sp_col, d.sp_val, d.w, d.lw, d.n_virt, p, d.tsum,
                                               dot ? d.sc : nullptr);
    }
    const SplitArgs a{d.sh_ptr, d.sh_col, d.sh_val, d.sl_mask, d.sl_first, d.cmb_ptr, d.cmb_slot, d.tsum};
    if (dot)
      k_spmv_split<true><<<row_grid(d), kRowThreads, 0, s>>>(a, d.w, d.lw, d.n_pad, p, q, d.part, d.sc);
    else
      k_spmv_split<false><<<row_grid(d), kRowThreads, 0, s>>>(a, d.w, d.lw, d.n_pad, p, q, d.part, d.sc);
    return;
  }
  if (d.vslice) {
    if (dot)
      k_spmv_vs<true><<<row_grid(d), kRowThreads, 0, s>>>(d.vs_c, d.vs_first, d.vs_ptr, d.vs_col, d.vs_val, d.w,
                                                          d.lw, d.n_pad, p, q, d.part, d.sc);
    else
      k_spmv_vs<false><<<row_grid(d), kRowThreads, 0, s>>>(d.vs_c, d.vs_first, d.vs_ptr, d.vs_col, d.vs_val, d.w,
                                                           d.lw, d.n_pad, p, q, d.part, d.sc);
    return;
  }
  enqueue_spmv_plain(d, p, q, dot, s);
}

void enqueue_spmv_plain(const DeviceLayout &d, const double *p, double *q, bool dot, cudaStream_t s) {
  if (spmv_tma_usable(d)) return enqueue_spmv_tma(d, p, q, dot, s);
  if (warp_spmv_usable(d)) return enqueue_spmv_warp(d, p, q, dot, s);
  if (dot)
    k_spmv<true><<<row_grid(d), kRowThreads, 0, s>>>(d.a_ptr, d.a_col, d.a_val, d.w, d.lw, d.n_pad, p, q, d.part, d.sc);
  else
    k_spmv<false><<<row_grid(d), kRowThreads, 0, s>>>(d.a_ptr, d.a_col, d.a_val, d.w, d.lw, d.n_pad, p, q, d.part, d.sc);
}

// Forward sweep over all colors: y (F64) or y32 (F32) from r.
// Colors pick their kernel one by one: the loader-thread kernel for colors
// with long other-color runs or few level-1 blocks, else the
// bulk-copy-staged warp kernel; both give the same bits.
int64_t sweep_launches(const DeviceLayout &d, int prec) { return dag_selected(d, prec) ? 1 : d.nc; }

int64_t precond_launches(const DeviceLayout &d, int prec) {
  return 2 * sweep_launches(d, prec) - (fb_tw_usable(d, prec) ? 1 : 0);
}

void enqueue_fwd(const DeviceLayout &d, int prec, const double *r, bool check_done, cudaStream_t s) {
  if (dag_selected(d, prec)) return enqueue_fwd_dag(d, prec, r, check_done, s);
  const bool wide = wide_usable(d, true, prec), tw = tw_usable(d, true, prec);
  if ((wide && wide_all(d)) || tw) {
    for (int c = 0; c < d.nc; ++c) {
      if (wide && wide_preferred(d, true, c)) launch_fwd_wide_color(d, prec, c, r, check_done, s);
      else launch_fwd_tw_color(d, prec, c, r, check_done, s);
    }
    return;
  }
  if (warp_usable(d, true, prec)) return enqueue_fwd_warp(d, prec, r, check_done, s);
  const Scalars *sc = check_done ? d.sc : nullptr;
  for (int c = 0; c < d.nc; ++c) {
    if (prec == HBMC_PREC_F64) {
      const SweepArgs<double> a = sweep_args<double>(d, true, c);
      k_fwd<double, double><<<sweep_grid(d, c), kTileThreads, sweep_smem(a), s>>>(a, r, d.y, sc);
    } else {
      const SweepArgs<float> a = sweep_args<float>(d, true, c);
      k_fwd<float, float><<<sweep_grid(d, c), kTileThreads, sweep_smem(a), s>>>(a, r, d.y32, sc);
    }
  }
}

// Backward sweep over all colors (n_c..1): z from y / y32; dot_mode 0: no
// dot, 1: initial rho = r.z, 2: rho and beta.
void enqueue_bwd(const DeviceLayout &d, int prec, const double *r, int dot_mode, bool check_done, cudaStream_t s) {
  if (dag_selected(d, prec)) return enqueue_bwd_dag(d, prec, r, dot_mode, check_done, s);
  const bool wide = wide_usable(d, false, prec), tw = tw_usable(d, false, prec);
  if ((wide && wide_all(d)) || tw) {
    auto use_wide = [&](int c) { return wide && wide_preferred(d, false, c); };
    int64_t total = 0;
    for (int c = 0; c < d.nc; ++c) total += use_wide(c) ? wide_color_grid(d, c) : tw_color_grid(d, c);
    int64_t off = 0;
    for (int c = d.nc - 1; c >= 0; --c) {
      if (use_wide(c)) {
        launch_bwd_wide_color(d, prec, c, r, dot_mode, check_done, off, c == 0, total, s);
        off += wide_color_grid(d, c);
      } else {
        launch_bwd_tw_color(d, prec, c, r, dot_mode, check_done, off, c == 0, total, s);
        off += tw_color_grid(d, c);
      }
    }
    return;
  }
  if (warp_usable(d, false, prec)) return enqueue_bwd_warp(d, prec, r, dot_mode, check_done, s);
  Scalars *sc = check_done || dot_mode ? d.sc : nullptr;
  int64_t total = 0;
  for (int c = 0; c < d.nc; ++c) total += sweep_grid(d, c);
  int64_t off = 0;
  for (int c = d.nc - 1; c >= 0; --c) {
    const unsigned grid = sweep_grid(d, c);
    const int last = c == 0;
    if (prec == HBMC_PREC_F64) {
      const SweepArgs<double> a = sweep_args<double>(d, false, c);
      k_bwd<double, double><<<grid, kTileThreads, sweep_smem(a), s>>>(a, d.y, d.z, d.z32, r, sc, dot_mode, d.part, off, last, total);
    } else {
      const SweepArgs<float> a = sweep_args<float>(d, false, c);
      k_bwd<float, float><<<grid, kTileThreads, sweep_smem(a), s>>>(a, d.y32, d.z, d.z32, r, sc, dot_mode, d.part, off, last, total);
    }
    off += grid;
  }
}

// ||b - A x|| / ||b|| of the context's b and x into the scalars' relres.
void enqueue_relres(const DeviceLayout &d, cudaStream_t s) {
  k_residual<0><<<row_grid(d), kRowThreads, 0, s>>>(
      d.a_ptr, d.a_col, d.a_val, d.w, d.lw, d.n_pad, d.b, d.x, d.r, d.part, d.sc, d.hist);
}

// z = M^{-1} r: the forward sweep over colors 1..n_c, then the backward
// sweep over n_c..1 (dot_mode as enqueue_bwd).  When the last color runs on
// the bulk-copy warp kernels in both directions, its forward and backward
// passes are one launch (k_fb_tw), with the same bits.
void enqueue_precond(const DeviceLayout &d, int prec, const double *r, int dot_mode, bool check_done,
                     cudaStream_t s) {
  if (!fb_tw_usable(d, prec)) {
    enqueue_fwd(d, prec, r, check_done, s);
    enqueue_bwd(d, prec, r, dot_mode, check_done, s);
    return;
  }
  const bool wide_f = wide_usable(d, true, prec), wide_b = wide_usable(d, false, prec);
  for (int c = 0; c < d.nc - 1; ++c) {
    if (wide_f && wide_preferred(d, true, c)) launch_fwd_wide_color(d, prec, c, r, check_done, s);
    else launch_fwd_tw_color(d, prec, c, r, check_done, s);
  }
  auto use_wide = [&](int c) { return wide_b && wide_preferred(d, false, c); };
  int64_t total = 0;
  for (int c = 0; c < d.nc; ++c) total += use_wide(c) ? wide_color_grid(d, c) : tw_color_grid(d, c);
  int64_t off = 0;
  launch_fb_tw_last(d, prec, r, dot_mode, check_done, off, d.nc == 1, total, s);
  off += tw_color_grid(d, d.nc - 1);
  for (int c = d.nc - 2; c >= 0; --c) {
    if (use_wide(c)) {
      launch_bwd_wide_color(d, prec, c, r, dot_mode, check_done, off, c == 0, total, s);
      off += wide_color_grid(d, c);
    } else {
      launch_bwd_tw_color(d, prec, c, r, dot_mode, check_done, off, c == 0, total, s);
      off += tw_color_grid(d, c);
    }
  }
}

// Before the loop: permute b and x0 in, r = b - A x, ||b||, z = M^{-1} r,
// rho = r.z, p = z.
void enqueue_init(const DeviceLayout &d, int prec, cudaStream_t s) {
  enqueue_gather_in(d, nullptr, d.b, 0, s);
  enqueue_gather_in(d, nullptr, d.x, 1, s);
  k_residual<0><<<row_grid(d), kRowThreads, 0, s>>>(
      d.a_ptr, d.a_col, d.a_val, d.w, d.lw, d.n_pad, d.b, d.x, d.r, d.part, d.sc, d.hist);
  enqueue_precond(d, prec, d.r, 1, true, s);
  k_update_p<<<row_grid(d), kRowThreads, 0, s>>>(d.n_pad, d.z, d.p, d.sc, 0, 0, 0);
}

// One CG iteration.
void enqueue_body(const DeviceLayout &d, int prec, cudaStream_t s, bool use_cond,
                  cudaGraphConditionalHandle h) {
  enqueue_spmv(d, d.p, d.q, true, s);
  k_update_xr<<<row_grid(d), kRowThreads, 0, s>>>(
      d.n_pad, d.p, d.q, d.x, d.r, d.part, d.sc, d.hist, use_cond ? 1 : 0, h);
  enqueue_precond(d, prec, d.r, 2, true, s);
  k_update_p<<<row_grid(d), kRowThreads, 0, s>>>(d.n_pad, d.z, d.p, d.sc, 1, use_cond ? 1 : 0, h);
}

void enqueue_update_xr(const DeviceLayout &d, cudaStream_t s) {
  k_update_xr<<<row_grid(d), kRowThreads, 0, s>>>(d.n_pad, d.p, d.q, d.x, d.r, d.part, d.sc, d.hist, 0, 0);
}

void enqueue_update_p(const DeviceLayout &d, cudaStream_t s) {
  k_update_p<<<row_grid(d), kRowThreads, 0, s>>>(d.n_pad, d.z, d.p, d.sc, 1, 0, 0);
}

// After the loop: x out, true residual.
void enqueue_final(const DeviceLayout &d, cudaStream_t s) {
  enqueue_gather_out(d, d.x, nullptr, true, s);
  k_residual<1><<<row_grid(d), kRowThreads, 0, s>>>(
      d.a_ptr, d.a_col, d.a_val, d.w, d.lw, d.n_pad, d.b, d.x, d.t, d.part, d.sc, d.hist);
}

void enqueue_reset_bad_row(const DeviceLayout &d, cudaStream_t s) { k_set_bad_row<<<1, 1, 0, s>>>(d.sc); }

void enqueue_ic0(const DeviceLayout &d, double shift, cudaStream_t s) {
  k_set_bad_row<<<1, 1, 0, s>>>(d.sc);
  for (int c = 0; c < d.nc; ++c) {
    const int64_t t0 = d.tile_ptr[c], nt = d.tile_ptr[c + 1] - t0;
    k_ic0<<<blocks_for(nt * d.w, kSweepThreads), kSweepThreads, 0, s>>>(
        d.lrp, d.lci, d.laval, d.adiag, 1.0 + shift, d.lval, d.ldiag, d.dinv, d.bs, d.w, t0, nt, d.sc);
  }
}

void enqueue_scatter_factor(const DeviceLayout &d, bool f32, cudaStream_t s, const double *bval) {
  if (!bval) bval = d.lval;
  if (d.nnz_lower > 0) {
    ScatterArgs a{d.lmap_f, d.lmap_b, d.lmapx_f, d.lmapx_b, d.fo_val, d.fi_val, d.bo_val, d.bi_val, d.fx_val,
                  d.bx_val, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    if (f32) {
      a.fo32 = d.fo_val32;
      a.fi32 = d.fi_val32;
      a.bo32 = d.bo_val32;
      a.bi32 = d.bi_val32;
      a.fx32 = d.fx_val32;
      a.bx32 = d.bx_val32;
    }
    k_scatter_factor<<<blocks_for(d.nnz_lower, kRowThreads), kRowThreads, 0, s>>>(d.nnz_lower, d.lval, bval, a);
  }
  if (f32) {
    enqueue_narrow(d.dinv, d.dinv32, d.n_pad, s);
    if (d.dinvb != d.dinv) enqueue_narrow(d.dinvb, d.dinvb32, d.n_pad, s);
  }
}

}  // namespace hbmc

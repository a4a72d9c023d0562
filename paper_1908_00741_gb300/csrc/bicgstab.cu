// ILU(0) and ILU(0)-preconditioned BiCGStab for matrices whose pattern is
// symmetric but whose values are not (Section 2: IC(0)/ILU(0)
// preconditioning; the HBMC ordering serves ILU(0)'s substitutions exactly
// as it serves IC(0)'s, with U in place of L^T).
//
// ILU(0) runs color by color like IC(0): lane j of a level-1 block owns BMC
// block j and walks its bs rows in order.  Row i, entries in ascending
// column:
//   w = abar_ij - sum_{k < min(i,j)} l_ik u_kj  (k ascending, one fma each),
//   l_ij = w / u_jj for j < i, u_ij = w for j >= i.
// u_kj (k < j) is kept at the strict-lower position of (j, k), so the same
// row-merge that finds l_jk for IC(0) finds u_kj here.  The forward sweep
// then multiplies by 1 (L is unit) and the backward sweep by 1 / u_ii.
//
// BiCGStab (right-preconditioned, van der Vorst) per iteration:
//   beta = (rho / rho_old)(alpha / omega); p = r + beta (p - omega v)
//   ph = M^{-1} p; v = A ph; alpha = rho / (rh, v); s = r - alpha v
//   (||s|| / ||b|| < tol: x += alpha ph, done); sh = M^{-1} s; t = A sh
//   omega = (t, s) / (t, t); x += alpha ph + omega sh; r = s - omega t
//   ||r|| / ||b|| < tol: done; rho_old = rho; rho = (rh, r)
// with the oracle's fused multiply-adds; every dot is a deterministic
// block tree finished by the grid's last block, which also applies the
// scalar step and the stopping tests, so the loop never returns to the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>

#include "device_util.cuh"
#include "hbmc_internal.h"
#include "kernels.h"

namespace hbmc {
namespace {

constexpr int kBThreads = 256;
constexpr int kBBlocksPerSm = 8;

inline unsigned bgrid(const DeviceLayout &d) {
  const int64_t full = (d.n_pad + kBThreads - 1) / kBThreads;
  const int64_t cap = (int64_t)d.sm_count * kBBlocksPerSm;
  return (unsigned)std::max<int64_t>(1, std::min(full, cap));
}

// ---------------------------------------------------------------------------
// ILU(0), one color
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128)
    k_ilu0(const int64_t *__restrict__ lrp, const int32_t *__restrict__ lci, const double *__restrict__ laval,
           const double *__restrict__ uaval, const double *__restrict__ adiag, const int64_t *__restrict__ urp,
           const int32_t *__restrict__ uci, const int64_t *__restrict__ upos, double scale, double *lval,
           double *uval, double *udiag, double *uinv, int bs, int w, int64_t tile0, int64_t ntiles, Scalars *sc) {
  if (sc->bad_row != LLONG_MAX) return;  // an earlier color failed
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tl = g / w;
  if (tl >= ntiles) return;
  const int j = (int)(g - tl * w);
  const int64_t s0 = (tile0 + tl) * bs;
  for (int l = 0; l < bs; ++l) {
    const int64_t i = (s0 + l) * w + j;
    const int64_t e0 = lrp[i], e1 = lrp[i + 1];
    // lower entries (i, c), c < i: l_ic = (a_ic - sum_{k<c} l_ik u_kc) / u_cc
    for (int64_t e = e0; e < e1; ++e) {
      const int64_t c = lci[e];
      double s = laval[e];
      int64_t p = e0, q = lrp[c];
      const int64_t qe = lrp[c + 1];
      while (p < e && q < qe) {
        const int32_t cp = lci[p], cq = lci[q];
        if (cp == cq) {
          s = fma(-lval[p], uval[q], s);
          ++p;
          ++q;
        } else if (cp < cq) {
          ++p;
        } else {
          ++q;
        }
      }
      lval[e] = s / udiag[c];
    }
    // pivot u_ii = (1 + shift) a_ii - sum_{k<i} l_ik u_ki
    double d = scale * adiag[i];
    for (int64_t e = e0; e < e1; ++e) d = fma(-lval[e], uval[e], d);
    if (d == 0.0 || !finite(d)) {
      atomicMin(&sc->bad_row, (long long)i);
      udiag[i] = nan("");
      uinv[i] = nan("");
      continue;
    }
    udiag[i] = d;
    uinv[i] = 1.0 / d;
    // upper entries (i, c), c > i: u_ic = a_ic - sum_{k<i} l_ik u_kc, stored
    // at the lower position of (c, i)
    for (int64_t f = urp[i]; f < urp[i + 1]; ++f) {
      const int64_t c = uci[f], pos = upos[f];
      double s = uaval[pos];
      int64_t p = e0, q = lrp[c];
      while (p < e1 && q < pos) {
        const int32_t cp = lci[p], cq = lci[q];
        if (cp == cq) {
          s = fma(-lval[p], uval[q], s);
          ++p;
          ++q;
        } else if (cp < cq) {
          ++p;
        } else {
          ++q;
        }
      }
      uval[pos] = s;
    }
  }
}

__global__ void k_fill(double *a, double v, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

// ---------------------------------------------------------------------------
// BiCGStab
// ---------------------------------------------------------------------------

// Deterministic sums over the grid of up to two per-thread values; true in
// every thread of the last block, which then holds the totals in thread 0.
template <int NV>
__device__ __forceinline__ bool grid_sums(const double (&v)[NV], double *part, unsigned *cnt, double (&out)[NV]) {
  double bsum[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) bsum[k] = block_sum<kBThreads>(v[k]);
  if (!publish(part + (size_t)NV * blockIdx.x, bsum, NV, cnt, gridDim.x)) return false;
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = gather_partials<kBThreads>(part, gridDim.x, NV, k);
  return true;
}

__device__ __forceinline__ void bcg_stop(Scalars *sc, int status) {
  sc->status = status;
  sc->done = 1;
}

// After r = b - A x0 (k_residual<0>): rh = r, p = v = 0, rho = (rh, r).
__global__ void __launch_bounds__(kBThreads)
    k_bcg_start(int64_t n_pad, const double *__restrict__ r, double *rh, double *p, double *v, double *part,
                Scalars *sc) {
  if (sc->done) return;
  double acc[1] = {0.0};
  FOR_ROWS(row, n_pad) {
    const double ri = r[row];
    rh[row] = ri;
    p[row] = 0.0;
    v[row] = 0.0;
    acc[0] = fma(ri, ri, acc[0]);
  }
  double tot[1];
  if (!grid_sums<1>(acc, part, &sc->cnt[CNT_RHO], tot) || threadIdx.x != 0) return;
  sc->cnt[CNT_RHO] = 0;
  sc->rho_old = 1.0;
  sc->alpha = 1.0;
  sc->omega = 1.0;
  sc->rho = tot[0];
  sc->half = 0;
  if (sc->maxit <= 0) return bcg_stop(sc, ST_MAXIT);
  if (tot[0] == 0.0 || !finite(tot[0])) bcg_stop(sc, ST_BREAKDOWN);
}

// p = r + beta (p - omega v)
__global__ void __launch_bounds__(kBThreads)
    k_bcg_p(int64_t n_pad, const double *__restrict__ r, const double *__restrict__ v, double *p,
            const Scalars *sc) {
  if (sc->done) return;
  const double beta = (sc->rho / sc->rho_old) * (sc->alpha / sc->omega), omega = sc->omega;
  FOR_ROWS(row, n_pad) p[row] = fma(beta, fma(-omega, v[row], p[row]), r[row]);
}

// alpha = rho / (rh, v)
__global__ void __launch_bounds__(kBThreads)
    k_bcg_alpha(int64_t n_pad, const double *__restrict__ rh, const double *__restrict__ v, double *part,
                Scalars *sc) {
  if (sc->done) return;
  double acc[1] = {0.0};
  FOR_ROWS(row, n_pad) acc[0] = fma(rh[row], v[row], acc[0]);
  double tot[1];
  if (!grid_sums<1>(acc, part, &sc->cnt[CNT_PQ], tot) || threadIdx.x != 0) return;
  sc->cnt[CNT_PQ] = 0;
  sc->rv = tot[0];
  if (tot[0] == 0.0 || !finite(tot[0])) return bcg_stop(sc, ST_BREAKDOWN);
  sc->alpha = sc->rho / tot[0];
}

// s = r - alpha v with ||s||; the half step may already meet the tolerance
__global__ void __launch_bounds__(kBThreads)
    k_bcg_s(int64_t n_pad, const double *__restrict__ r, const double *__restrict__ v, double *s, double *part,
            Scalars *sc, double *hist) {
  if (sc->done) return;
  const double alpha = sc->alpha;
  double acc[1] = {0.0};
  FOR_ROWS(row, n_pad) {
    const double si = fma(-alpha, v[row], r[row]);
    s[row] = si;
    acc[0] = fma(si, si, acc[0]);
  }
  double tot[1];
  if (!grid_sums<1>(acc, part, &sc->cnt[CNT_S], tot) || threadIdx.x != 0) return;
  sc->cnt[CNT_S] = 0;
  const double res = sqrt(tot[0]) / sc->bnorm;
  if (res < sc->tol) {
    const long long k = sc->iters + 1;
    sc->iters = k;
    sc->relres = res;
    if (k < kHistCap) hist[k] = res;
    sc->half = 1;
    bcg_stop(sc, ST_CONVERGED);
  }
}

// omega = (t, s) / (t, t)
__global__ void __launch_bounds__(kBThreads)
    k_bcg_omega(int64_t n_pad, const double *__restrict__ t, const double *__restrict__ s, double *part,
                Scalars *sc) {
  if (sc->done) return;
  double acc[2] = {0.0, 0.0};
  FOR_ROWS(row, n_pad) {
    const double ti = t[row];
    acc[0] = fma(ti, ti, acc[0]);
    acc[1] = fma(ti, s[row], acc[1]);
  }
  double tot[2];
  if (!grid_sums<2>(acc, part, &sc->cnt[CNT_W], tot) || threadIdx.x != 0) return;
  sc->cnt[CNT_W] = 0;
  sc->tt = tot[0];
  sc->ts = tot[1];
  if (!(tot[0] > 0.0) || !finite(tot[0])) return bcg_stop(sc, ST_BREAKDOWN);
  sc->omega = tot[1] / tot[0];
}

// x += alpha ph + omega sh, r = s - omega t, ||r|| and the stopping tests,
// then rho_old = rho, rho = (rh, r).  After a half step that met the
// tolerance only x += alpha ph and r = s remain.
__global__ void __launch_bounds__(kBThreads)
    k_bcg_xr(int64_t n_pad, const double *__restrict__ ph, const double *__restrict__ sh,
             const double *__restrict__ t, const double *__restrict__ s, const double *__restrict__ rh, double *x,
             double *r, double *part, Scalars *sc, double *hist, int use_cond, cudaGraphConditionalHandle handle) {
  if (sc->done) {
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(handle, 0);
    if (!sc->half) return;
    const double alpha = sc->alpha;
    FOR_ROWS(row, n_pad) {
      x[row] = fma(alpha, ph[row], x[row]);
      r[row] = s[row];
    }
    // once: the last block clears the flag (every block has read it by then)
    if (publish(nullptr, nullptr, 0, &sc->cnt[CNT_S], gridDim.x) && threadIdx.x == 0) {
      sc->cnt[CNT_S] = 0;
      sc->half = 0;
    }
    return;
  }
  const double alpha = sc->alpha, omega = sc->omega;
  double acc[2] = {0.0, 0.0};
  FOR_ROWS(row, n_pad) {
    x[row] = fma(omega, sh[row], fma(alpha, ph[row], x[row]));
    const double ri = fma(-omega, t[row], s[row]);
    r[row] = ri;
    acc[0] = fma(ri, ri, acc[0]);
    acc[1] = fma(rh[row], ri, acc[1]);
  }
  double tot[2];
  if (!grid_sums<2>(acc, part, &sc->cnt[CNT_RR], tot) || threadIdx.x != 0) return;
  sc->cnt[CNT_RR] = 0;
  const long long k = sc->iters + 1;
  sc->iters = k;
  const double res = sqrt(tot[0]) / sc->bnorm;
  sc->relres = res;
  if (k < kHistCap) hist[k] = res;
  if (res < sc->tol) bcg_stop(sc, ST_CONVERGED);
  else if (omega == 0.0 || !finite(omega)) bcg_stop(sc, ST_BREAKDOWN);
  else if (k >= sc->maxit) bcg_stop(sc, ST_MAXIT);
  else {
    sc->rho_old = sc->rho;
    sc->rho = tot[1];
    if (tot[1] == 0.0 || !finite(tot[1])) bcg_stop(sc, ST_BREAKDOWN);
  }
  if (sc->done && use_cond) cudaGraphSetConditional(handle, 0);
}

}  // namespace

void enqueue_ilu0(const DeviceLayout &d, double shift, cudaStream_t s) {
  enqueue_reset_bad_row(d, s);
  for (int c = 0; c < d.nc; ++c) {
    const int64_t t0 = d.tile_ptr[c], nt = d.tile_ptr[c + 1] - t0;
    const int64_t threads = nt * d.w;
    k_ilu0<<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(d.lrp, d.lci, d.laval, d.uaval, d.adiag, d.urp, d.uci,
                                                              d.upos, 1.0 + shift, d.lval, d.uval, d.udiag, d.dinvb,
                                                              d.bs, d.w, t0, nt, d.sc);
  }
}

void enqueue_unit_dinv(const DeviceLayout &d, cudaStream_t s) {
  k_fill<<<(unsigned)((d.n_pad + 255) / 256), 256, 0, s>>>(d.dinv, 1.0, d.n_pad);
}

void enqueue_bcg_init(const DeviceLayout &d, cudaStream_t s) {
  enqueue_gather_in(d, nullptr, d.b, 0, s);
  enqueue_gather_in(d, nullptr, d.x, 1, s);
  enqueue_relres(d, s);
  k_bcg_start<<<bgrid(d), kBThreads, 0, s>>>(d.n_pad, d.r, d.rh, d.p, d.q, d.part, d.sc);
}

// One BiCGStab iteration: v lives in q, s in sv, ph in ph, sh in z, t in t.
cudaError_t enqueue_bcg_body(const DeviceLayout &d, int prec, cudaStream_t s, bool use_cond,
                             cudaGraphConditionalHandle h) {
  const unsigned g = bgrid(d);
  const size_t bytes = sizeof(double) * (size_t)d.n_pad;
  k_bcg_p<<<g, kBThreads, 0, s>>>(d.n_pad, d.r, d.q, d.p, d.sc);
  enqueue_fwd(d, prec, d.p, true, s);
  enqueue_bwd(d, prec, nullptr, 0, true, s);
  cudaError_t e = cudaMemcpyAsync(d.ph, d.z, bytes, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  enqueue_spmv_plain(d, d.ph, d.q, false, s);
  k_bcg_alpha<<<g, kBThreads, 0, s>>>(d.n_pad, d.rh, d.q, d.part, d.sc);
  k_bcg_s<<<g, kBThreads, 0, s>>>(d.n_pad, d.r, d.q, d.sv, d.part, d.sc, d.hist);
  enqueue_fwd(d, prec, d.sv, true, s);
  enqueue_bwd(d, prec, nullptr, 0, true, s);
  enqueue_spmv_plain(d, d.z, d.t, false, s);
  k_bcg_omega<<<g, kBThreads, 0, s>>>(d.n_pad, d.t, d.sv, d.part, d.sc);
  k_bcg_xr<<<g, kBThreads, 0, s>>>(d.n_pad, d.ph, d.z, d.t, d.sv, d.rh, d.x, d.r, d.part, d.sc, d.hist,
                                   use_cond ? 1 : 0, h);
  return cudaGetLastError();
}

int64_t bcg_partials_needed(const DeviceLayout &d) { return 2 * (int64_t)bgrid(d) + 64; }

}  // namespace hbmc

// The whole IC(0)-CG solve as one persistent cooperative kernel (w = 32).
//
// Every CUDA block stays resident for the solve (cooperative launch, one
// block per SM).  The phases of a CG iteration -- SpMV with p.q, the x/r
// update with ||r||, the forward sweep color by color, the backward sweep
// color by color with r.z, the p update -- are separated by grid-wide
// barriers instead of kernel boundaries, which is what a small system
// needs: at 32^3 a color has 64 level-1 blocks and the launches, not the
// work, set the time.  The n_c - 1 synchronizations per sweep of Section
// 4.3.3 are these barriers.
//
// The arithmetic of each phase is the graph path's: the row SpMV and the
// warp-per-level-1-block sweeps with the layout's term order, so SpMV, both
// substitutions and the vector updates give the oracle's bits.  Dot
// products: each block sums its threads' terms with the fixed block tree,
// writes one partial, and after the barrier every block adds the partials
// in block order -- the same values in every block, so every block takes the
// same scalar steps and stopping decision without another barrier.
//
// Data written by one block and read by another in a later phase is read
// with plain coherent loads after the barrier's fences (never through the
// read-only path).  Every barrier wait is bounded: a block that waits too
// long raises an error flag, every block then leaves, and the solve reports
// a timeout.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>

#include "device_util.cuh"
#include "hbmc_internal.h"
#include "kernels.h"
#include "warp_common.cuh"

namespace hbmc {
namespace {

constexpr int kPWarps = 8;
constexpr int kPThreads = 32 * kPWarps;
constexpr long long kBarSpins = 1ll << 28;  // polls of an L2 line: seconds before giving up

template <typename T>
struct PArgs {
  // SpMV
  const int64_t *a_ptr;
  const int32_t *a_col;
  const double *a_val;
  // sweeps: [0] forward, [1] backward
  const int32_t *rec[2];
  const int32_t *o_col[2];
  const uint8_t *i_m[2];
  const T *o_val[2];
  const T *i_val[2];
  const T *dinv[2];
  uint32_t off_t[2], off_d[2], off_iv[2], off_im[2], warp_bytes[2];
  const int64_t *tile_ptr;  // device copy, nc + 1
  int rec_ints, bs, nc;
  int64_t n_pad;
  // vectors
  const double *b;
  double *x, *r, *z, *p, *q;
  T *y;        // forward result (y or its FP32 twin)
  float *z32;  // FP32 copy of z (FP32 sweeps)
  double *part, *hist;
  unsigned *bar;  // [0] arrivals, [1] generation, [2] error flag
};

// Grid-wide barrier; false once any block gave up waiting.
__device__ __forceinline__ bool gsync(unsigned *bar) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = bar + 1;
    volatile unsigned *err = bar + 2;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      bar[0] = 0;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*gen == g && !*err) {
        if (++spins > kBarSpins) {
          atomicExch(bar + 2, 1u);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile unsigned *)(bar + 2) == 0;
}

// Sum of the blocks' partials (slot k of nv per block), same in every block.
__device__ __forceinline__ double sum_partials(const double *part, int nv, int k) {
  double acc = 0.0;
  for (int64_t b = threadIdx.x; b < gridDim.x; b += kPThreads) acc += __ldcg(part + b * nv + k);
  return block_sum<kPThreads>(acc);  // valid in thread 0
}

__device__ __forceinline__ double bcast(double v) {
  __shared__ double s;
  __syncthreads();
  if (threadIdx.x == 0) s = v;
  __syncthreads();
  return s;
}

__device__ __forceinline__ double sell_row_p(const int64_t *a_ptr, const int32_t *a_col, const double *a_val,
                                             int64_t row, const double *v) {
  const int64_t s = row >> 5;
  const int j = (int)(row & 31);
  const int64_t pe = a_ptr[s + 1];
  double acc = 0.0;
  for (int64_t e = a_ptr[s] + j; e < pe; e += 32) acc = fma(a_val[e], v[a_col[e]], acc);
  return acc;
}

// One level-1 block of a sweep by one warp (the warp-per-unit kernels' steps).
template <typename T, bool FWD>
__device__ __forceinline__ void p_unit(const PArgs<T> &a, unsigned char *ws, int64_t u, int lane, double &rz) {
  constexpr int D = FWD ? 0 : 1;
  int32_t *rs = reinterpret_cast<int32_t *>(ws);
  T *ts = reinterpret_cast<T *>(ws + a.off_t[D]);
  T *ds = reinterpret_cast<T *>(ws + a.off_d[D]);
  T *iv = reinterpret_cast<T *>(ws + a.off_iv[D]);
  uint8_t *im = ws + a.off_im[D];
  const int bs = a.bs;
  const int64_t row0 = u * (int64_t)bs * 32;
  const int32_t *rc = a.rec[D] + u * a.rec_ints;
  for (int k = lane; k < a.rec_ints; k += 32) rs[k] = rc[k];
  for (int l = 0; l < bs; ++l) {
    const int64_t row = row0 + (l << 5) + lane;
    ts[(l << 5) + lane] = FWD ? (T)a.r[row] : (T)a.y[row];
    ds[(l << 5) + lane] = a.dinv[D][row];
  }
  __syncwarp();
  const int ilen = rs[1];
  const int64_t ibeg = rec64(rs, 4);
  for (int e = lane; e < ilen; e += 32) {
    iv[e] = a.i_val[D][ibeg + e];
    im[e] = a.i_m[D][ibeg + e];
  }
  __syncwarp();
  // other-color couplings, in run order (kChunk loads in flight per lane)
  {
    const int olen = rs[0];
    const int64_t obeg = rec64(rs, 2);
    const int32_t *rel = rs + 6;
    int l = 0;
    for (int t0 = 0; t0 < olen; t0 += kChunk * 32) {
      int32_t c[kChunk];
      T v[kChunk], g[kChunk];
#pragma unroll
      for (int k = 0; k < kChunk; ++k) {
        const int t = t0 + k * 32;
        if (t < olen) {
          c[k] = a.o_col[D][obeg + t + lane];
          v[k] = a.o_val[D][obeg + t + lane];
        }
      }
#pragma unroll
      for (int k = 0; k < kChunk; ++k) {
        const int t = t0 + k * 32;
        if (t < olen) {
          if constexpr (FWD) g[k] = a.y[c[k]];
          else if constexpr (sizeof(T) == 4) g[k] = (T)a.z32[c[k]];
          else g[k] = (T)a.z[c[k]];
        }
      }
#pragma unroll
      for (int k = 0; k < kChunk; ++k) {
        const int t = t0 + k * 32;
        if (t < olen) {
          while (t >= rel[l + 1]) ++l;
          T *slot = ts + (l << 5) + lane;
          *slot = fma(-v[k], g[k], *slot);
        }
      }
    }
  }
  const int32_t *i_rel = rs + 7 + bs;
  for (int q = 0; q < bs; ++q) {
    const int l = FWD ? q : bs - 1 - q;
    T acc = ts[(l << 5) + lane];
    const int pe = i_rel[l + 1];
    for (int p = i_rel[l] + lane; p < pe; p += 32) acc = fma(-iv[p], ts[(im[p] << 5) + lane], acc);
    ts[(l << 5) + lane] = acc * ds[(l << 5) + lane];
  }
  for (int l = 0; l < bs; ++l) {
    const int64_t row = row0 + (l << 5) + lane;
    const T v = ts[(l << 5) + lane];
    if constexpr (FWD) {
      a.y[row] = v;
    } else {
      a.z[row] = (double)v;
      if constexpr (sizeof(T) == 4) a.z32[row] = v;
      rz = fma(a.r[row], (double)v, rz);
    }
  }
  __syncwarp();
}

// The preconditioner z = M^{-1} r; returns r.z (same in every block) or
// NaN when a barrier gave up.
template <typename T>
__device__ double p_precond(const PArgs<T> &a, unsigned char *smem) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * kPWarps + warp, nw = (int64_t)gridDim.x * kPWarps;
  for (int c = 0; c < a.nc; ++c) {
    double unused = 0.0;
    for (int64_t u = a.tile_ptr[c] + gw; u < a.tile_ptr[c + 1]; u += nw)
      p_unit<T, true>(a, smem + (size_t)warp * a.warp_bytes[0], u, lane, unused);
    if (!gsync(a.bar)) return nan("");
  }
  double rz = 0.0;
  for (int c = a.nc - 1; c >= 0; --c) {
    for (int64_t u = a.tile_ptr[c] + gw; u < a.tile_ptr[c + 1]; u += nw)
      p_unit<T, false>(a, smem + (size_t)warp * a.warp_bytes[1], u, lane, rz);
    if (c > 0 && !gsync(a.bar)) return nan("");
  }
  const double v = block_sum<kPThreads>(rz);
  if (threadIdx.x == 0) a.part[blockIdx.x] = v;
  if (!gsync(a.bar)) return nan("");
  return bcast(sum_partials(a.part, 1, 0));
}

template <typename T>
__global__ void __launch_bounds__(kPThreads, 1) k_cg_persistent(const PArgs<T> a, Scalars *sc) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int64_t n = a.n_pad;
  const int64_t t0 = (int64_t)blockIdx.x * kPThreads + threadIdx.x, nt = (int64_t)gridDim.x * kPThreads;
  const double tol = sc->tol;
  const long long maxit = sc->maxit;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  int status = ST_RUNNING;
  long long k = 0;
  double res = 0.0, bnorm = 0.0;
  // r = b - A x, ||b||, ||r||
  {
    double bb = 0.0, rr = 0.0;
    for (int64_t row = t0; row < n; row += nt) {
      const double acc = sell_row_p(a.a_ptr, a.a_col, a.a_val, row, a.x);
      const double bi = a.b[row], ri = bi - acc;
      a.r[row] = ri;
      bb = fma(bi, bi, bb);
      rr = fma(ri, ri, rr);
    }
    const double vb = block_sum<kPThreads>(bb), vr = block_sum<kPThreads>(rr);
    if (threadIdx.x == 0) {
      a.part[2 * blockIdx.x] = vb;
      a.part[2 * blockIdx.x + 1] = vr;
    }
    if (!gsync(a.bar)) goto timeout;
    const double sbb = bcast(sum_partials(a.part, 2, 0)), srr = bcast(sum_partials(a.part, 2, 1));
    bnorm = sqrt(sbb);
    if (bnorm == 0.0) {
      for (int64_t row = t0; row < n; row += nt) a.x[row] = 0.0;
      if (lead) {
        sc->zero_x = 1;
        a.hist[0] = 0.0;
      }
      status = ST_CONVERGED;
      goto finish;
    }
    res = sqrt(srr) / bnorm;
    if (lead) a.hist[0] = res;
    if (res < tol) {
      status = ST_CONVERGED;
      goto finish;
    }
    if (maxit <= 0) {
      status = ST_MAXIT;
      goto finish;
    }
  }
  {
    double rho = p_precond<T>(a, smem);
    if (rho != rho) goto timeout;
    if (!(rho > 0.0) || !finite(rho)) {
      status = ST_BREAKDOWN;
      goto finish;
    }
    for (int64_t row = t0; row < n; row += nt) a.p[row] = a.z[row];
    if (!gsync(a.bar)) goto timeout;
    for (k = 1;; ++k) {
      // q = A p, p.q
      double pq = 0.0;
      for (int64_t row = t0; row < n; row += nt) {
        const double acc = sell_row_p(a.a_ptr, a.a_col, a.a_val, row, a.p);
        a.q[row] = acc;
        pq = fma(a.p[row], acc, pq);
      }
      {
        const double v = block_sum<kPThreads>(pq);
        if (threadIdx.x == 0) a.part[blockIdx.x] = v;
      }
      if (!gsync(a.bar)) goto timeout;
      const double spq = bcast(sum_partials(a.part, 1, 0));
      if (!(spq > 0.0) || !finite(spq)) {
        --k;
        status = ST_BREAKDOWN;
        break;
      }
      const double alpha = rho / spq;
      // x += alpha p, r -= alpha q, ||r||
      double rr = 0.0;
      for (int64_t row = t0; row < n; row += nt) {
        a.x[row] = fma(alpha, a.p[row], a.x[row]);
        const double ri = fma(-alpha, a.q[row], a.r[row]);
        a.r[row] = ri;
        rr = fma(ri, ri, rr);
      }
      {
        const double v = block_sum<kPThreads>(rr);
        if (threadIdx.x == 0) a.part[blockIdx.x] = v;
      }
      if (!gsync(a.bar)) goto timeout;
      res = sqrt(bcast(sum_partials(a.part, 1, 0))) / bnorm;
      if (lead && k < kHistCap) a.hist[k] = res;
      if (res < tol) {
        status = ST_CONVERGED;
        break;
      }
      if (k >= maxit) {
        status = ST_MAXIT;
        break;
      }
      const double rho_new = p_precond<T>(a, smem);
      if (rho_new != rho_new) goto timeout;
      if (!(rho_new > 0.0) || !finite(rho_new)) {
        status = ST_BREAKDOWN;
        break;
      }
      const double beta = rho_new / rho;
      rho = rho_new;
      for (int64_t row = t0; row < n; row += nt) a.p[row] = fma(beta, a.p[row], a.z[row]);
      if (!gsync(a.bar)) goto timeout;
    }
  }
finish:
  if (lead) {
    sc->iters = k;
    sc->relres = bnorm == 0.0 ? 0.0 : res;
    sc->bnorm = bnorm;
    sc->status = status;
    sc->done = 1;
  }
  return;
timeout:
  if (lead) {
    sc->timeout = 1;
    sc->iters = k;
    sc->status = ST_BREAKDOWN;
    sc->done = 1;
  }
}

template <typename T>
PArgs<T> p_args(const DeviceLayout &d, int prec) {
  PArgs<T> a;
  a.a_ptr = d.a_ptr;
  a.a_col = d.a_col;
  a.a_val = d.a_val;
  for (int D = 0; D < 2; ++D) {
    const bool fwd = D == 0;
    a.rec[D] = fwd ? d.rec_f : d.rec_b;
    a.o_col[D] = fwd ? d.fo_col : d.bo_col;
    a.i_m[D] = fwd ? d.fi_m : d.bi_m;
    if constexpr (sizeof(T) == 8) {
      a.o_val[D] = (const T *)(fwd ? d.fo_val : d.bo_val);
      a.i_val[D] = (const T *)(fwd ? d.fi_val : d.bi_val);
      a.dinv[D] = (const T *)(fwd ? d.dinv : d.dinvb);
    } else {
      a.o_val[D] = (const T *)(fwd ? d.fo_val32 : d.bo_val32);
      a.i_val[D] = (const T *)(fwd ? d.fi_val32 : d.bi_val32);
      a.dinv[D] = (const T *)(fwd ? d.dinv32 : d.dinvb32);
    }
    const WarpPlan &w = prec == HBMC_PREC_F64 ? (fwd ? d.wp_f64_f : d.wp_f64_b) : (fwd ? d.wp_f32_f : d.wp_f32_b);
    a.off_t[D] = w.off_t;
    a.off_d[D] = w.off_d;
    a.off_iv[D] = w.off_iv;
    a.off_im[D] = w.off_im;
    a.warp_bytes[D] = w.warp_bytes;
  }
  a.tile_ptr = d.tile_ptr_dev;
  a.rec_ints = d.rec_ints;
  a.bs = d.bs;
  a.nc = d.nc;
  a.n_pad = d.n_pad;
  a.b = d.b;
  a.x = d.x;
  a.r = d.r;
  a.z = d.z;
  a.p = d.p;
  a.q = d.q;
  if constexpr (sizeof(T) == 8) a.y = (T *)d.y;
  else a.y = (T *)d.y32;
  a.z32 = d.z32;
  a.part = d.part;
  a.hist = d.hist;
  a.bar = d.pbar;
  return a;
}

size_t p_smem(const DeviceLayout &d, int prec) {
  const WarpPlan &f = prec == HBMC_PREC_F64 ? d.wp_f64_f : d.wp_f32_f;
  const WarpPlan &b = prec == HBMC_PREC_F64 ? d.wp_f64_b : d.wp_f32_b;
  return (size_t)kPWarps * std::max(f.warp_bytes, b.warp_bytes);
}

constexpr size_t kPSmemBudget = 200 * 1024;

}  // namespace

cudaError_t setup_persistent() {
  cudaError_t e = cudaFuncSetAttribute(k_cg_persistent<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kPSmemBudget);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_cg_persistent<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kPSmemBudget);
}

bool persistent_usable(const DeviceLayout &d, int prec) {
  return d.w == 32 && !d.split && d.rec_f && d.tile_ptr_dev && d.pbar && p_smem(d, prec) <= kPSmemBudget &&
         d.part_len >= 2 * (int64_t)d.sm_count;
}

// The solve after the permutation in: one cooperative launch.
cudaError_t enqueue_persistent(const DeviceLayout &d, int prec, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(d.pbar, 0, 4 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  const size_t sm = p_smem(d, prec);
  dim3 grid((unsigned)d.sm_count), block(kPThreads);
  if (prec == HBMC_PREC_F64) {
    PArgs<double> a = p_args<double>(d, prec);
    Scalars *sc = d.sc;
    void *args[] = {&a, &sc};
    return cudaLaunchCooperativeKernel((const void *)k_cg_persistent<double>, grid, block, args, sm, s);
  }
  PArgs<float> a = p_args<float>(d, prec);
  Scalars *sc = d.sc;
  void *args[] = {&a, &sc};
  return cudaLaunchCooperativeKernel((const void *)k_cg_persistent<float>, grid, block, args, sm, s);
}

}  // namespace hbmc

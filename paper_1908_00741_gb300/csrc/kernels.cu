// CUDA kernels of the HBMC-ICCG solve (sm_103a) and the sequences that
// enqueue them.
//
// Thread mapping of the substitutions (Section 4.2.2, Eqs. "BAMC3", "y2-2",
// "y2-3"): one group of w consecutive threads per level-1 block, lane j owns
// BMC block j of that level-1 block, and the bs steps run in order inside the
// thread.  Step l of all w lanes touches w consecutive rows, so every slice
// column of the SELL layout is one coalesced load.  Couplings to other colors
// are independent of the step chain and are gathered for all bs steps first;
// the chain itself only involves the lane's own earlier steps and runs out of
// shared memory.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>

#include "hbmc_internal.h"
#include "kernels.h"

namespace hbmc {
namespace {

constexpr int kRowThreads = 256;
constexpr int kSweepThreads = 128;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum (fixed butterfly and tree); valid in thread 0.
template <int NT>
__device__ double block_sum(double v) {
  __shared__ double red[NT / 32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (wid == 0) {
    s = lane < NT / 32 ? red[lane] : 0.0;
    s = warp_sum(s);
  }
  return s;
}

// Thread 0 stores the block's partial(s); returns true in every thread of
// the last block of the grid to arrive.
__device__ bool publish(double *slot, const double *vals, int nv, unsigned *cnt, unsigned nblocks) {
  __shared__ unsigned s_last;
  if (threadIdx.x == 0) {
    for (int k = 0; k < nv; ++k) slot[k] = vals[k];
    __threadfence();
    const unsigned t = atomicAdd(cnt, 1u);
    s_last = (t == nblocks - 1);
  }
  __syncthreads();
  return s_last != 0;
}

// Sum of part[k * stride + off] for k < count, in a fixed order; valid in thread 0.
template <int NT>
__device__ double gather_partials(const double *part, int64_t count, int stride, int off) {
  __threadfence();
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < count; k += NT) acc += __ldcg(part + k * stride + off);
  return block_sum<NT>(acc);
}

__device__ __forceinline__ bool finite(double v) { return isfinite(v); }

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
                                           const double *__restrict__ a_val, int w, int64_t row,
                                           const double *x) {
  const int64_t s = row / w;
  const int j = (int)(row - s * w);
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
               const double *__restrict__ a_val, int w, int64_t n_pad, const double *b,
               const double *x, double *r, double *part, Scalars *sc, double *hist) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double bb = 0.0, rr = 0.0;
  if (row < n_pad) {
    const double acc = sell_row(a_ptr, a_col, a_val, w, row, x);
    const double bi = b[row];
    const double ri = bi - acc;
    if (kMode == 0) r[row] = ri;
    bb = bi * bi;
    rr = ri * ri;
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
           const double *__restrict__ a_val, int w, int64_t n_pad, const double *p, double *q,
           double *part, Scalars *sc) {
  if (kDot && sc->done) return;
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double pq = 0.0;
  if (row < n_pad) {
    const double acc = sell_row(a_ptr, a_col, a_val, w, row, p);
    q[row] = acc;
    pq = p[row] * acc;
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
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double rr = 0.0;
  if (row < n_pad) {
    x[row] = fma(alpha, p[row], x[row]);
    const double ri = fma(-alpha, q[row], r[row]);
    r[row] = ri;
    rr = ri * ri;
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
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n_pad) return;
  p[row] = mode == 0 ? z[row] : fma(sc->beta, p[row], z[row]);
}

// ---------------------------------------------------------------------------
// Forward substitution, one color (Eqs. "for2", "for3", "y2-2", "y2-3"):
//   y_i = (r_i - sum_j l_ij y_j) * dinv_i
// T: arithmetic of the factor and of the accumulation; Y: storage of y.
// ---------------------------------------------------------------------------
template <typename T, typename Y>
__global__ void __launch_bounds__(kSweepThreads)
    k_fwd(const int64_t *__restrict__ fo_ptr, const int32_t *__restrict__ fo_col,
          const T *__restrict__ fo_val, const int64_t *__restrict__ fi_ptr,
          const uint8_t *__restrict__ fi_m, const T *__restrict__ fi_val,
          const T *__restrict__ dinv, const double *__restrict__ r, Y *y, int bs, int w,
          int64_t tile0, int64_t ntiles, const Scalars *sc) {
  extern __shared__ unsigned char smem_raw[];
  T *ts = reinterpret_cast<T *>(smem_raw);  // [bs][blockDim]: t_l, then y_l
  if (sc && sc->done) return;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tl = g / w;
  if (tl >= ntiles) return;
  const int j = (int)(g - tl * w);
  const int64_t s0 = (tile0 + tl) * bs;
  const int nt = blockDim.x, me = threadIdx.x;
  // couplings to earlier colors: independent of the step chain
  for (int l = 0; l < bs; ++l) {
    const int64_t s = s0 + l;
    T acc = (T)r[s * w + j];
    const int64_t pe = fo_ptr[s + 1];
    for (int64_t p = fo_ptr[s] + j; p < pe; p += w) acc = fma(-fo_val[p], (T)y[fo_col[p]], acc);
    ts[l * nt + me] = acc;
  }
  // the bs-step chain of this lane's BMC block
  for (int l = 0; l < bs; ++l) {
    const int64_t s = s0 + l;
    const int64_t row = s * w + j;
    T acc = ts[l * nt + me];
    const int64_t pe = fi_ptr[s + 1];
    for (int64_t p = fi_ptr[s] + j; p < pe; p += w) acc = fma(-fi_val[p], ts[fi_m[p] * nt + me], acc);
    const T yv = acc * dinv[row];
    ts[l * nt + me] = yv;
    y[row] = (Y)yv;
  }
}

// ---------------------------------------------------------------------------
// Backward substitution, one color (Section 4.2.2, last paragraph):
//   z_i = (y_i - sum_j l_ji z_j) * dinv_i, steps bs..1
// Optionally accumulates r.z for the CG (dot_mode 1: initial rho, 2: rho and
// beta inside the loop); the launch of the last color finishes the sum.
// ---------------------------------------------------------------------------
template <typename T, typename Y>
__global__ void __launch_bounds__(kSweepThreads)
    k_bwd(const int64_t *__restrict__ bo_ptr, const int32_t *__restrict__ bo_col,
          const T *__restrict__ bo_val, const int64_t *__restrict__ bi_ptr,
          const uint8_t *__restrict__ bi_m, const T *__restrict__ bi_val,
          const T *__restrict__ dinv, const Y *__restrict__ yin, double *z,
          const double *__restrict__ r, int bs, int w, int64_t tile0, int64_t ntiles,
          Scalars *sc, int dot_mode, double *part, int64_t part_off, int last_launch,
          int64_t part_total) {
  extern __shared__ unsigned char smem_raw[];
  T *ts = reinterpret_cast<T *>(smem_raw);
  if (sc && sc->done) return;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tl = g / w;
  const bool active = tl < ntiles;
  const int j = (int)(g - tl * w);
  const int64_t s0 = (tile0 + tl) * bs;
  const int nt = blockDim.x, me = threadIdx.x;
  double rz = 0.0;
  if (active) {
    for (int l = 0; l < bs; ++l) {
      const int64_t s = s0 + l;
      T acc = (T)yin[s * w + j];
      const int64_t pe = bo_ptr[s + 1];
      for (int64_t p = bo_ptr[s] + j; p < pe; p += w) acc = fma(-bo_val[p], (T)z[bo_col[p]], acc);
      ts[l * nt + me] = acc;
    }
    for (int l = bs - 1; l >= 0; --l) {
      const int64_t s = s0 + l;
      const int64_t row = s * w + j;
      T acc = ts[l * nt + me];
      const int64_t pe = bi_ptr[s + 1];
      for (int64_t p = bi_ptr[s] + j; p < pe; p += w) acc = fma(-bi_val[p], ts[bi_m[p] * nt + me], acc);
      const T zv = acc * dinv[row];
      ts[l * nt + me] = zv;
      z[row] = (double)zv;
      if (dot_mode) rz = fma(r[row], (double)zv, rz);
    }
  }
  if (!dot_mode) return;
  double v = block_sum<kSweepThreads>(rz);
  if (threadIdx.x == 0) part[part_off + blockIdx.x] = v;
  if (!last_launch) return;
  // the last color's launch: all earlier colors' partials are complete
  __shared__ unsigned s_last;
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(&sc->cnt[CNT_RZ], 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  const double rho_new = gather_partials<kSweepThreads>(part, part_total, 1, 0);
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
__global__ void k_scatter_factor(int64_t nnz_lower, const double *__restrict__ lval,
                                 const int64_t *__restrict__ lmap_f,
                                 const int64_t *__restrict__ lmap_b, double *fo, double *fi,
                                 double *bo, double *bi, float *fo32, float *fi32, float *bo32,
                                 float *bi32) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz_lower) return;
  const double v = lval[e];
  const int64_t f = lmap_f[e], b = lmap_b[e];
  if (f >= 0) fo[f] = v; else fi[-f - 1] = v;
  if (b >= 0) bo[b] = v; else bi[-b - 1] = v;
  if (fo32) {
    if (f >= 0) fo32[f] = (float)v; else fi32[-f - 1] = (float)v;
    if (b >= 0) bo32[b] = (float)v; else bi32[-b - 1] = (float)v;
  }
}

__global__ void k_set_bad_row(Scalars *sc) {
  sc->bad_row = LLONG_MAX;
  sc->done = 0;
}

inline unsigned blocks_for(int64_t n, int nt) { return (unsigned)((n + nt - 1) / nt); }

template <typename T>
size_t sweep_smem(int bs) { return (size_t)bs * kSweepThreads * sizeof(T); }

}  // namespace

// ---------------------------------------------------------------------------
// Enqueue sequences
// ---------------------------------------------------------------------------

cudaError_t setup_kernels() {
  cudaError_t e = cudaSuccess;
  const int f64 = (int)(kMaxBs * kSweepThreads * sizeof(double));
  const int f32 = (int)(kMaxBs * kSweepThreads * sizeof(float));
  if ((e = cudaFuncSetAttribute(k_fwd<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, f64))) return e;
  if ((e = cudaFuncSetAttribute(k_bwd<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, f64))) return e;
  if ((e = cudaFuncSetAttribute(k_fwd<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, f32))) return e;
  if ((e = cudaFuncSetAttribute(k_bwd<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, f32))) return e;
  return e;
}

int64_t partials_needed(const DeviceLayout &d) {
  int64_t sweep = 0;
  for (int c = 0; c < d.nc; ++c)
    sweep += blocks_for((d.tile_ptr[c + 1] - d.tile_ptr[c]) * d.w, kSweepThreads);
  const int64_t rows = 2 * (int64_t)blocks_for(d.n_pad, kRowThreads);
  return (sweep > rows ? sweep : rows) + 64;
}

void enqueue_gather_in(const DeviceLayout &d, const double *src, double *dst, int which, cudaStream_t s) {
  k_gather_in<<<blocks_for(d.n_pad, kRowThreads), kRowThreads, 0, s>>>(src, dst, d.inv, d.n_pad, d.sc, which);
}

void enqueue_gather_out(const DeviceLayout &d, const double *src, double *dst, bool to_user, cudaStream_t s) {
  k_gather_out<<<blocks_for(d.n, kRowThreads), kRowThreads, 0, s>>>(src, dst, d.pi, d.n, to_user ? d.sc : nullptr);
}

void enqueue_widen(const float *src, double *dst, int64_t n, cudaStream_t s) {
  k_widen<<<blocks_for(n, kRowThreads), kRowThreads, 0, s>>>(src, dst, n);
}

void enqueue_narrow(const double *src, float *dst, int64_t n, cudaStream_t s) {
  k_narrow<<<blocks_for(n, kRowThreads), kRowThreads, 0, s>>>(src, dst, n);
}

void enqueue_spmv(const DeviceLayout &d, const double *p, double *q, bool dot, cudaStream_t s) {
  if (dot)
    k_spmv<true><<<blocks_for(d.n_pad, kRowThreads), kRowThreads, 0, s>>>(d.a_ptr, d.a_col, d.a_val, d.w, d.n_pad, p, q, d.part, d.sc);
  else
    k_spmv<false><<<blocks_for(d.n_pad, kRowThreads), kRowThreads, 0, s>>>(d.a_ptr, d.a_col, d.a_val, d.w, d.n_pad, p, q, d.part, d.sc);
}

// Forward sweep over all colors: y (F64) or y32 (F32) from r.
void enqueue_fwd(const DeviceLayout &d, int prec, const double *r, bool check_done, cudaStream_t s) {
  const Scalars *sc = check_done ? d.sc : nullptr;
  for (int c = 0; c < d.nc; ++c) {
    const int64_t t0 = d.tile_ptr[c], nt = d.tile_ptr[c + 1] - t0;
    const unsigned grid = blocks_for(nt * d.w, kSweepThreads);
    if (prec == HBMC_PREC_F64)
      k_fwd<double, double><<<grid, kSweepThreads, sweep_smem<double>(d.bs), s>>>(
          d.fo_ptr, d.fo_col, d.fo_val, d.fi_ptr, d.fi_m, d.fi_val, d.dinv, r, d.y, d.bs, d.w, t0, nt, sc);
    else
      k_fwd<float, float><<<grid, kSweepThreads, sweep_smem<float>(d.bs), s>>>(
          d.fo_ptr, d.fo_col, d.fo_val32, d.fi_ptr, d.fi_m, d.fi_val32, d.dinv32, r, d.y32, d.bs, d.w, t0, nt, sc);
  }
}

// Backward sweep over all colors (n_c..1): z from y / y32; dot_mode 0: no
// dot, 1: initial rho = r.z, 2: rho and beta.
void enqueue_bwd(const DeviceLayout &d, int prec, const double *r, int dot_mode, bool check_done, cudaStream_t s) {
  Scalars *sc = check_done || dot_mode ? d.sc : nullptr;
  int64_t total = 0;
  for (int c = 0; c < d.nc; ++c) total += blocks_for((d.tile_ptr[c + 1] - d.tile_ptr[c]) * d.w, kSweepThreads);
  int64_t off = 0;
  for (int c = d.nc - 1; c >= 0; --c) {
    const int64_t t0 = d.tile_ptr[c], nt = d.tile_ptr[c + 1] - t0;
    const unsigned grid = blocks_for(nt * d.w, kSweepThreads);
    const int last = c == 0;
    if (prec == HBMC_PREC_F64)
      k_bwd<double, double><<<grid, kSweepThreads, sweep_smem<double>(d.bs), s>>>(
          d.bo_ptr, d.bo_col, d.bo_val, d.bi_ptr, d.bi_m, d.bi_val, d.dinv, d.y, d.z, r, d.bs, d.w,
          t0, nt, sc, dot_mode, d.part, off, last, total);
    else
      k_bwd<float, float><<<grid, kSweepThreads, sweep_smem<float>(d.bs), s>>>(
          d.bo_ptr, d.bo_col, d.bo_val32, d.bi_ptr, d.bi_m, d.bi_val32, d.dinv32, d.y32, d.z, r,
          d.bs, d.w, t0, nt, sc, dot_mode, d.part, off, last, total);
    off += grid;
  }
}

// Before the loop: permute b and x0 in, r = b - A x, ||b||, z = M^{-1} r,
// rho = r.z, p = z.
void enqueue_init(const DeviceLayout &d, int prec, cudaStream_t s) {
  enqueue_gather_in(d, nullptr, d.b, 0, s);
  enqueue_gather_in(d, nullptr, d.x, 1, s);
  k_residual<0><<<blocks_for(d.n_pad, kRowThreads), kRowThreads, 0, s>>>(
      d.a_ptr, d.a_col, d.a_val, d.w, d.n_pad, d.b, d.x, d.r, d.part, d.sc, d.hist);
  enqueue_fwd(d, prec, d.r, true, s);
  enqueue_bwd(d, prec, d.r, 1, true, s);
  k_update_p<<<blocks_for(d.n_pad, kRowThreads), kRowThreads, 0, s>>>(d.n_pad, d.z, d.p, d.sc, 0, 0, 0);
}

// One CG iteration.
void enqueue_body(const DeviceLayout &d, int prec, cudaStream_t s, bool use_cond,
                  cudaGraphConditionalHandle h) {
  enqueue_spmv(d, d.p, d.q, true, s);
  k_update_xr<<<blocks_for(d.n_pad, kRowThreads), kRowThreads, 0, s>>>(
      d.n_pad, d.p, d.q, d.x, d.r, d.part, d.sc, d.hist, use_cond ? 1 : 0, h);
  enqueue_fwd(d, prec, d.r, true, s);
  enqueue_bwd(d, prec, d.r, 2, true, s);
  k_update_p<<<blocks_for(d.n_pad, kRowThreads), kRowThreads, 0, s>>>(d.n_pad, d.z, d.p, d.sc, 1, use_cond ? 1 : 0, h);
}

// After the loop: x out, true residual.
void enqueue_final(const DeviceLayout &d, cudaStream_t s) {
  enqueue_gather_out(d, d.x, nullptr, true, s);
  k_residual<1><<<blocks_for(d.n_pad, kRowThreads), kRowThreads, 0, s>>>(
      d.a_ptr, d.a_col, d.a_val, d.w, d.n_pad, d.b, d.x, d.t, d.part, d.sc, d.hist);
}

void enqueue_ic0(const DeviceLayout &d, double shift, cudaStream_t s) {
  k_set_bad_row<<<1, 1, 0, s>>>(d.sc);
  for (int c = 0; c < d.nc; ++c) {
    const int64_t t0 = d.tile_ptr[c], nt = d.tile_ptr[c + 1] - t0;
    k_ic0<<<blocks_for(nt * d.w, kSweepThreads), kSweepThreads, 0, s>>>(
        d.lrp, d.lci, d.laval, d.adiag, 1.0 + shift, d.lval, d.ldiag, d.dinv, d.bs, d.w, t0, nt, d.sc);
  }
}

void enqueue_scatter_factor(const DeviceLayout &d, bool f32, cudaStream_t s) {
  if (d.nnz_lower > 0)
    k_scatter_factor<<<blocks_for(d.nnz_lower, kRowThreads), kRowThreads, 0, s>>>(
        d.nnz_lower, d.lval, d.lmap_f, d.lmap_b, d.fo_val, d.fi_val, d.bo_val, d.bi_val,
        f32 ? d.fo_val32 : nullptr, f32 ? d.fi_val32 : nullptr, f32 ? d.bo_val32 : nullptr,
        f32 ? d.bi_val32 : nullptr);
  if (f32) enqueue_narrow(d.dinv, d.dinv32, d.n_pad, s);
}

}  // namespace hbmc

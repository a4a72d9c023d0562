// Batched HBMC-ICCG: many independent SPD systems, one launch per color.
//
// The batch is one block-diagonal system laid out color-major (batch_host.cpp),
// so the warp-per-level-1-block kernels sweep every system's units of a color
// in a single launch.  What differs from the single-system solve is the CG
// control: every system has its own scalars (rho, alpha, beta, ||b||), its
// own stopping test and its own iteration count.  Each kernel that feeds a
// dot product writes one partial per level-1 block (a warp's sum over its
// rows); a finishing kernel with one CUDA block per system then adds the
// partials of that system in a fixed order and updates its scalars.  Systems
// that are done are skipped by every later kernel; the CG loop (a CUDA graph
// while node, as for one system) ends when no system is left running.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "device_util.cuh"
#include "hbmc.h"
#include "hbmc_internal.h"
#include "kernels.h"
#include "warp_common.cuh"

namespace hbmc {
namespace {

struct BSys {
  double rho, beta, alpha, bnorm, relres, true_relres;
  long long iters;
  int status, done, zero_x, pad;
  unsigned long long t_done;
};

struct BGlob {
  double tol;
  long long maxit;
  int active;     // systems still running
  unsigned cnt;   // arrival counter of the finishing kernels
  unsigned long long t0;
  const double *user_b;
  double *user_x;
};

enum { F_INIT = 0, F_PQ = 1, F_RR = 2, F_RZ_INIT = 3, F_RZ = 4, F_TRUE = 5 };
constexpr int kFinishThreads = 256;
constexpr int kBWpb = 4;

__device__ __forceinline__ bool sys_done(const BSys *bs, const int32_t *unit_sys, int64_t u) {
  return bs[unit_sys[u]].done != 0;
}

// ---------------------------------------------------------------------------
// permutations
// ---------------------------------------------------------------------------
__global__ void k_bgather_in(double *dst, const int32_t *__restrict__ inv, int64_t n_pad, BGlob *bg, int which) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (which == 0 && k == 0) bg->t0 = global_ns();
  if (k >= n_pad) return;
  const double *src = which == 0 ? bg->user_b : bg->user_x;
  const int32_t i = inv[k];
  dst[k] = i >= 0 ? src[i] : 0.0;
}

__global__ void k_bgather_out(const double *src, const int32_t *__restrict__ pi, int64_t n,
                              const int32_t *__restrict__ unit_sys, int64_t R, const BSys *bsys, BGlob *bg) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t k = pi[i];
  bg->user_x[i] = bsys[unit_sys[k / R]].zero_x ? 0.0 : src[k];
}

// ---------------------------------------------------------------------------
// SpMV-shaped kernels, W lanes per level-1 block (w = W): a warp holds 32 / W
// level-1 blocks.  Work is predicated, not skipped by early returns, so that
// every lane reaches the per-level-1-block reductions.
// ---------------------------------------------------------------------------
template <int W>
struct Lanes {
  static constexpr int kPerWarp = 32 / W;
  int sub, j;  // level-1 block within the warp, lane within the level-1 block
  unsigned mask;
  __device__ Lanes(int lane)
      : sub(lane / W), j(lane % W), mask(W == 32 ? 0xffffffffu : (0xffffu << (16 * (lane / W)))) {}
};

// sum over the W lanes of a level-1 block (every lane of the warp calls it)
template <int W>
__device__ __forceinline__ double unit_sum(double v) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct ARun {
  const int32_t *rec;
  int rec_ints;
  const int32_t *col;
  const double *val;
  int bs;
  int64_t units;
  uint32_t off_t, unit_bytes;
  // the variable-slice-height layout (vs_c null: the plain one)
  const uint8_t *vs_c;
  const int64_t *vs_first, *vs_ptr;
  const int32_t *vs_col;
  const double *vs_val;
  int lw;
};

template <int W>
__device__ __forceinline__ int64_t unit_of(int warp, const Lanes<W> &ln) {
  return ((int64_t)blockIdx.x * kBWpb + warp) * Lanes<W>::kPerWarp + ln.sub;
}

template <int W>
__device__ __forceinline__ double *spmv_unit(const ARun &a, unsigned char *smem, int warp, const Lanes<W> &ln,
                                             int64_t u, const double *x) {
  unsigned char *ws = smem + (size_t)(warp * Lanes<W>::kPerWarp + ln.sub) * a.unit_bytes;
  int32_t *rs = reinterpret_cast<int32_t *>(ws);
  double *ts = reinterpret_cast<double *>(ws + a.off_t);
  const int32_t *rc = a.rec + u * a.rec_ints;
  for (int k = ln.j; k < a.rec_ints; k += W) rs[k] = rc[k];
  if (a.vs_c) {
    // every lane its own rows of the variable-height layout (same sums)
    for (int l = 0; l < a.bs; ++l)
      ts[l * W + ln.j] = vs_row(a.vs_c, a.vs_first, a.vs_ptr, a.vs_col, a.vs_val, W, a.lw,
                                (u * a.bs + l) * W + ln.j, x);
    __syncwarp(ln.mask);
    return ts;
  }
  for (int l = 0; l < a.bs; ++l) ts[l * W + ln.j] = 0.0;
  __syncwarp(ln.mask);
  run_accumulate<double, double, false, W>(a.col, a.val, x, rec64(rs, 2), rs[0], rs + 6, ts, ln.j);
  return ts;
}

// mode 0: r = b - A x with ||b||^2 -> part0, ||r||^2 -> part1 (every system);
// mode 1: ||b - A x||^2 -> part0 (true residual after the loop).
template <int kMode, int W>
__global__ void __launch_bounds__(32 * kBWpb)
    k_bresid_w(const ARun a, const double *b, const double *x, double *r, double *part0, double *part1) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5;
  const Lanes<W> ln(threadIdx.x & 31);
  const int64_t u = unit_of<W>(warp, ln);
  double bb = 0.0, rr = 0.0;
  if (u < a.units) {
    const double *ts = spmv_unit<W>(a, smem, warp, ln, u, x);
    const int64_t row0 = u * (int64_t)a.bs * W;
    for (int l = 0; l < a.bs; ++l) {
      const int64_t row = row0 + l * W + ln.j;
      const double bi = b[row];
      const double ri = bi - ts[l * W + ln.j];
      if (kMode == 0) r[row] = ri;
      bb = fma(bi, bi, bb);
      rr = fma(ri, ri, rr);
    }
  }
  bb = unit_sum<W>(bb);
  rr = unit_sum<W>(rr);
  if (u < a.units && ln.j == 0) {
    if (kMode == 0) {
      part0[u] = bb;
      part1[u] = rr;
    } else {
      part0[u] = rr;
    }
  }
}

template <int W>
__global__ void __launch_bounds__(32 * kBWpb)
    k_bspmv_w(const ARun a, const int32_t *__restrict__ unit_sys, const BSys *bsys, const double *p, double *q,
              double *part0) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5;
  const Lanes<W> ln(threadIdx.x & 31);
  const int64_t u = unit_of<W>(warp, ln);
  const bool live = u < a.units && !sys_done(bsys, unit_sys, u);
  double pq = 0.0;
  if (live) {
    const double *ts = spmv_unit<W>(a, smem, warp, ln, u, p);
    const int64_t row0 = u * (int64_t)a.bs * W;
    for (int l = 0; l < a.bs; ++l) {
      const int64_t row = row0 + l * W + ln.j;
      const double qv = ts[l * W + ln.j];
      q[row] = qv;
      pq = fma(p[row], qv, pq);
    }
  }
  pq = unit_sum<W>(pq);
  if (u < a.units && ln.j == 0) part0[u] = live ? pq : 0.0;
}

// x += alpha_s p, r -= alpha_s q, ||r||^2 partial
template <int W>
__global__ void __launch_bounds__(32 * kBWpb)
    k_bupdate_xr_w(int bs, int64_t units, const int32_t *__restrict__ unit_sys, const BSys *bsys, const double *p,
                   const double *q, double *x, double *r, double *part0) {
  const int warp = threadIdx.x >> 5;
  const Lanes<W> ln(threadIdx.x & 31);
  const int64_t u = unit_of<W>(warp, ln);
  const bool live = u < units && !sys_done(bsys, unit_sys, u);
  double rr = 0.0;
  if (live) {
    const double alpha = bsys[unit_sys[u]].alpha;
    const int64_t row0 = u * (int64_t)bs * W;
    for (int l = 0; l < bs; ++l) {
      const int64_t row = row0 + l * W + ln.j;
      x[row] = fma(alpha, p[row], x[row]);
      const double ri = fma(-alpha, q[row], r[row]);
      r[row] = ri;
      rr = fma(ri, ri, rr);
    }
  }
  rr = unit_sum<W>(rr);
  if (u < units && ln.j == 0) part0[u] = live ? rr : 0.0;
}

// p = z (mode 0) or p = z + beta_s p (mode 1)
template <int W>
__global__ void __launch_bounds__(32 * kBWpb)
    k_bupdate_p_w(int bs, int64_t units, const int32_t *__restrict__ unit_sys, const BSys *bsys, const double *z,
                  double *p, int mode) {
  const int warp = threadIdx.x >> 5;
  const Lanes<W> ln(threadIdx.x & 31);
  const int64_t u = unit_of<W>(warp, ln);
  if (u >= units) return;  // no reduction follows
  const BSys &s = bsys[unit_sys[u]];
  if (s.done) return;
  const double beta = s.beta;
  const int64_t row0 = u * (int64_t)bs * W;
  for (int l = 0; l < bs; ++l) {
    const int64_t row = row0 + l * W + ln.j;
    p[row] = mode == 0 ? z[row] : fma(beta, p[row], z[row]);
  }
}

// ---------------------------------------------------------------------------
// substitutions (same arithmetic as the single-system warp kernels)
// ---------------------------------------------------------------------------
template <typename T>
struct BSweep {
  const int32_t *rec;
  const int32_t *o_col;
  const T *o_val;
  const uint8_t *i_m;
  const T *i_val;
  const T *dinv;
  int bs, rec_ints;
  int64_t tile0, ntiles;
  uint32_t off_t, off_d, off_iv, off_im, unit_bytes;
};

template <typename T, typename IN, int W>
__device__ __forceinline__ T *stage(const BSweep<T> &a, unsigned char *smem, int warp, const Lanes<W> &ln,
                                    int64_t u, const IN *in, int32_t *&rs, T *&ds, T *&iv, uint8_t *&im) {
  unsigned char *ws = smem + (size_t)(warp * Lanes<W>::kPerWarp + ln.sub) * a.unit_bytes;
  rs = reinterpret_cast<int32_t *>(ws);
  T *ts = reinterpret_cast<T *>(ws + a.off_t);
  ds = reinterpret_cast<T *>(ws + a.off_d);
  iv = reinterpret_cast<T *>(ws + a.off_iv);
  im = ws + a.off_im;
  const int32_t *rc = a.rec + u * a.rec_ints;
  for (int k = ln.j; k < a.rec_ints; k += W) rs[k] = rc[k];
  const int64_t row0 = u * (int64_t)a.bs * W;
  for (int l = 0; l < a.bs; ++l) {
    const int64_t row = row0 + l * W + ln.j;
    ts[l * W + ln.j] = (T)in[row];
    ds[l * W + ln.j] = a.dinv[row];
  }
  __syncwarp(ln.mask);
  const int ilen = rs[1];
  const int64_t ibeg = rec64(rs, 4);
  for (int e = ln.j; e < ilen; e += W) {
    iv[e] = a.i_val[ibeg + e];
    im[e] = a.i_m[ibeg + e];
  }
  __syncwarp(ln.mask);
  return ts;
}

template <typename T, typename Y, int W>
__global__ void __launch_bounds__(32 * kBWpb)
    k_bfwd_w(const BSweep<T> a, const int32_t *__restrict__ unit_sys, const BSys *bsys, const double *__restrict__ r,
             Y *y) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5;
  const Lanes<W> ln(threadIdx.x & 31);
  const int64_t u = a.tile0 + unit_of<W>(warp, ln);
  if (u >= a.tile0 + a.ntiles || sys_done(bsys, unit_sys, u)) return;  // no reduction follows
  int32_t *rs;
  T *ds, *iv;
  uint8_t *im;
  T *ts = stage<T, double, W>(a, smem, warp, ln, u, r, rs, ds, iv, im);
  run_accumulate<T, Y, true, W>(a.o_col, a.o_val, y, rec64(rs, 2), rs[0], rs + 6, ts, ln.j);
  const int32_t *i_rel = rs + 7 + a.bs;
  for (int l = 0; l < a.bs; ++l) {
    T acc = ts[l * W + ln.j];
    const int pe = i_rel[l + 1];
    for (int p = i_rel[l] + ln.j; p < pe; p += W) acc = fma(-iv[p], ts[im[p] * W + ln.j], acc);
    ts[l * W + ln.j] = acc * ds[l * W + ln.j];
  }
  Y *yo = y + u * (int64_t)a.bs * W;
  for (int l = 0; l < a.bs; ++l) yo[l * W + ln.j] = (Y)ts[l * W + ln.j];
}

template <typename T, typename Y, int W>
__global__ void __launch_bounds__(32 * kBWpb)
    k_bbwd_w(const BSweep<T> a, const int32_t *__restrict__ unit_sys, const BSys *bsys, const Y *__restrict__ yin,
             double *z, const double *__restrict__ r, int dot, double *part0) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5;
  const Lanes<W> ln(threadIdx.x & 31);
  const int64_t u = a.tile0 + unit_of<W>(warp, ln);
  const bool in_range = u < a.tile0 + a.ntiles;
  const bool live = in_range && !sys_done(bsys, unit_sys, u);
  double rz = 0.0;
  if (live) {
    int32_t *rs;
    T *ds, *iv;
    uint8_t *im;
    T *ts = stage<T, Y, W>(a, smem, warp, ln, u, yin, rs, ds, iv, im);
    run_accumulate<T, double, true, W>(a.o_col, a.o_val, z, rec64(rs, 2), rs[0], rs + 6, ts, ln.j);
    const int32_t *i_rel = rs + 7 + a.bs;
    for (int l = a.bs - 1; l >= 0; --l) {
      T acc = ts[l * W + ln.j];
      const int pe = i_rel[l + 1];
      for (int p = i_rel[l] + ln.j; p < pe; p += W) acc = fma(-iv[p], ts[im[p] * W + ln.j], acc);
      ts[l * W + ln.j] = acc * ds[l * W + ln.j];
    }
    const int64_t row0 = u * (int64_t)a.bs * W;
    for (int l = 0; l < a.bs; ++l) {
      const double zv = (double)ts[l * W + ln.j];
      z[row0 + l * W + ln.j] = zv;
      if (dot) rz = fma(r[row0 + l * W + ln.j], zv, rz);
    }
  }
  if (!dot) return;  // uniform over the launch
  rz = unit_sum<W>(rz);
  if (in_range && ln.j == 0) part0[u] = live ? rz : 0.0;
}

// ---------------------------------------------------------------------------
// per-system finishing: one CUDA block per system
// ---------------------------------------------------------------------------
__device__ void become_done(BSys &s, BGlob *bg, int status) {
  s.status = status;
  s.done = 1;
  s.t_done = global_ns();
  atomicSub(&bg->active, 1);
}

template <int kMode>
__global__ void __launch_bounds__(kFinishThreads)
    k_bfinish(int32_t nsys, int32_t nc, const int64_t *__restrict__ cu_start, const int64_t *__restrict__ cu_count,
              const double *part0, const double *part1, BSys *bsys, BGlob *bg, int use_cond,
              cudaGraphConditionalHandle handle) {
  const int s = blockIdx.x;
  double a0 = 0.0, a1 = 0.0;
  for (int c = 0; c < nc; ++c) {
    const int64_t u0 = cu_start[(int64_t)s * nc + c], cnt = cu_count[(int64_t)s * nc + c];
    for (int64_t k = threadIdx.x; k < cnt; k += kFinishThreads) {
      a0 += part0[u0 + k];
      if (kMode == F_INIT) a1 += part1[u0 + k];
    }
  }
  const double s0 = block_sum_rt(a0);
  const double s1 = kMode == F_INIT ? block_sum_rt(a1) : 0.0;
  if (threadIdx.x == 0) {
    BSys &y = bsys[s];
    if (kMode == F_INIT) {
      y.iters = 0;
      y.bnorm = sqrt(s0);
      if (y.bnorm == 0.0) {
        y.zero_x = 1;
        y.relres = 0.0;
        become_done(y, bg, ST_CONVERGED);
      } else {
        y.relres = sqrt(s1) / y.bnorm;
        if (y.relres < bg->tol) become_done(y, bg, ST_CONVERGED);
        else if (bg->maxit <= 0) become_done(y, bg, ST_MAXIT);
      }
    } else if (kMode == F_TRUE) {
      y.true_relres = y.bnorm > 0.0 ? sqrt(s0) / y.bnorm : 0.0;
    } else if (!y.done) {
      if (kMode == F_PQ) {
        if (!(s0 > 0.0) || !finite(s0)) become_done(y, bg, ST_BREAKDOWN);
        else y.alpha = y.rho / s0;
      } else if (kMode == F_RR) {
        y.iters += 1;
        y.relres = sqrt(s0) / y.bnorm;
        if (y.relres < bg->tol) become_done(y, bg, ST_CONVERGED);
        else if (y.iters >= bg->maxit) become_done(y, bg, ST_MAXIT);
      } else {  // F_RZ_INIT, F_RZ
        if (!(s0 > 0.0) || !finite(s0)) {
          become_done(y, bg, ST_BREAKDOWN);
        } else {
          if (kMode == F_RZ) y.beta = s0 / y.rho;
          y.rho = s0;
        }
      }
    }
  }
  if (!use_cond) return;
  __shared__ unsigned last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&bg->cnt, 1u) == (unsigned)nsys - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    bg->cnt = 0;
    __threadfence();
    if (atomicAdd(&bg->active, 0) <= 0) cudaGraphSetConditional(handle, 0);
  }
}

// ---------------------------------------------------------------------------
// IC(0) with a shift per system
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128)
    k_bic0(const int64_t *__restrict__ lrp, const int32_t *__restrict__ lci, const double *__restrict__ laval,
           const double *__restrict__ adiag, const double *__restrict__ scale, const int32_t *__restrict__ unit_sys,
           double *lval, double *ldiag, double *dinv, int bs, int w, int64_t tile0, int64_t ntiles,
           long long *bad) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tl = g / w;
  if (tl >= ntiles) return;
  const int j = (int)(g % w);
  const int64_t u = tile0 + tl;
  const int32_t s = unit_sys[u];
  if (bad[s] != LLONG_MAX) return;  // this system failed in an earlier color
  const double sc = scale[s];
  for (int l = 0; l < bs; ++l) {
    const int64_t i = (u * bs + l) * w + j;
    const int64_t e0 = lrp[i], e1 = lrp[i + 1];
    for (int64_t e = e0; e < e1; ++e) {
      const int64_t jj = lci[e];
      double v = laval[e];
      int64_t p = e0, q = lrp[jj];
      const int64_t qe = lrp[jj + 1];
      while (p < e && q < qe) {
        const int32_t cp = lci[p], cq = lci[q];
        if (cp == cq) {
          v = fma(-lval[p], lval[q], v);
          ++p;
          ++q;
        } else if (cp < cq) {
          ++p;
        } else {
          ++q;
        }
      }
      lval[e] = v / ldiag[jj];
    }
    double d = sc * adiag[i];
    for (int64_t e = e0; e < e1; ++e) d = fma(-lval[e], lval[e], d);
    if (!(d > 0.0) || !finite(d)) {
      atomicMin(&bad[s], (long long)i);
      ldiag[i] = nan("");
      dinv[i] = nan("");
      continue;
    }
    const double ld = sqrt(d);
    ldiag[i] = ld;
    dinv[i] = 1.0 / ld;
  }
}

__global__ void k_fill_ll(long long *p, int64_t n, long long v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace
}  // namespace hbmc

// ===========================================================================
// host side
// ===========================================================================
using hbmc::BGlob;
using hbmc::BSys;
using hbmc::DeviceLayout;

struct hbmc_batch {
  hbmc_ctx *ctx = nullptr;
  hbmc::BatchMeta meta;
  std::string err;
  int32_t precision = HBMC_PREC_F64;
  int32_t loop_mode = HBMC_LOOP_GRAPH;
  int32_t check_every = 16;
  bool factored = false;
  int32_t *unit_sys = nullptr;
  int64_t *cu_start = nullptr, *cu_count = nullptr;
  BSys *bsys = nullptr;
  BGlob *bg = nullptr;
  double *part0 = nullptr, *part1 = nullptr, *scale = nullptr;
  long long *bad = nullptr;
  BSys *h_bsys = nullptr;
  BGlob *h_bg = nullptr;
  cudaStream_t cap[2] = {nullptr, nullptr};
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  std::vector<void *> allocs;
};

namespace {

thread_local std::string g_batch_err;

hbmc_status berr(hbmc_batch *b, hbmc_status s, const std::string &m) {
  if (b) b->err = m; else g_batch_err = m;
  return s;
}

#define BCK(call)                                                                                   \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      return berr(b, e_ == cudaErrorMemoryAllocation ? HBMC_ERR_OOM : HBMC_ERR_CUDA,                \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                              \
  } while (0)

struct View {
  const DeviceLayout *d;
  cudaStream_t s;
  int dev;
};

bool view(hbmc_batch *b, View &v) {
  bool factored;
  std::string *e;
  return hbmc::ctx_view(b->ctx, &v.d, &v.s, &v.dev, &factored, &e);
}

template <class T>
hbmc_status balloc(hbmc_batch *b, T *&p, size_t count) {
  void *q = nullptr;
  BCK(cudaMalloc(&q, (count ? count : 1) * sizeof(T)));
  b->allocs.push_back(q);
  BCK(cudaMemset(q, 0, (count ? count : 1) * sizeof(T)));
  p = static_cast<T *>(q);
  return HBMC_OK;
}

template <class T>
hbmc_status bupload(hbmc_batch *b, T *&p, const std::vector<T> &v) {
  hbmc_status s = balloc(b, p, v.size());
  if (s != HBMC_OK) return s;
  if (!v.empty()) BCK(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return HBMC_OK;
}

hbmc::ARun arun(const DeviceLayout &d) {
  hbmc::ARun a;
  a.rec = d.rec_a;
  a.rec_ints = d.rec_ints;
  a.col = d.a_col;
  a.val = d.a_val;
  a.bs = d.bs;
  a.units = d.tile_ptr[d.nc];
  a.off_t = d.wp_spmv.off_t;
  a.unit_bytes = d.wp_spmv.warp_bytes;
  a.vs_c = d.vslice ? d.vs_c : nullptr;
  a.vs_first = d.vs_first;
  a.vs_ptr = d.vs_ptr;
  a.vs_col = d.vs_col;
  a.vs_val = d.vs_val;
  a.lw = d.lw;
  return a;
}

template <typename T>
hbmc::BSweep<T> bsweep(const DeviceLayout &d, bool fwd, int c) {
  const hbmc::WarpPlan &w = sizeof(T) == 8 ? (fwd ? d.wp_f64_f : d.wp_f64_b) : (fwd ? d.wp_f32_f : d.wp_f32_b);
  hbmc::BSweep<T> a;
  a.rec = fwd ? d.rec_f : d.rec_b;
  a.o_col = fwd ? d.fo_col : d.bo_col;
  a.i_m = fwd ? d.fi_m : d.bi_m;
  if constexpr (sizeof(T) == 8) {
    a.o_val = (const T *)(fwd ? d.fo_val : d.bo_val);
    a.i_val = (const T *)(fwd ? d.fi_val : d.bi_val);
    a.dinv = (const T *)d.dinv;
  } else {
    a.o_val = (const T *)(fwd ? d.fo_val32 : d.bo_val32);
    a.i_val = (const T *)(fwd ? d.fi_val32 : d.bi_val32);
    a.dinv = (const T *)d.dinv32;
  }
  a.bs = d.bs;
  a.rec_ints = d.rec_ints;
  a.tile0 = d.tile_ptr[c];
  a.ntiles = d.tile_ptr[c + 1] - d.tile_ptr[c];
  a.off_t = w.off_t;
  a.off_d = w.off_d;
  a.off_iv = w.off_iv;
  a.off_im = w.off_im;
  a.unit_bytes = w.warp_bytes;
  return a;
}

// level-1 blocks per warp and per CUDA block of the batched kernels
int per_warp(const DeviceLayout &d) { return 32 / d.w; }
int64_t per_block(const DeviceLayout &d) { return (int64_t)hbmc::kBWpb * per_warp(d); }

size_t sweep_smem(const DeviceLayout &d, bool fwd, int prec) {
  const hbmc::WarpPlan &w = prec == HBMC_PREC_F64 ? (fwd ? d.wp_f64_f : d.wp_f64_b) : (fwd ? d.wp_f32_f : d.wp_f32_b);
  return (size_t)per_block(d) * w.warp_bytes;
}

template <int W>
void enq_fwd_w(hbmc_batch *b, const DeviceLayout &d, int prec, cudaStream_t s) {
  for (int c = 0; c < d.nc; ++c) {
    const unsigned grid = hbmc::nblk(d.tile_ptr[c + 1] - d.tile_ptr[c], (int)per_block(d));
    if (prec == HBMC_PREC_F64)
      hbmc::k_bfwd_w<double, double, W><<<grid, 32 * hbmc::kBWpb, sweep_smem(d, true, prec), s>>>(
          bsweep<double>(d, true, c), b->unit_sys, b->bsys, d.r, d.y);
    else
      hbmc::k_bfwd_w<float, float, W><<<grid, 32 * hbmc::kBWpb, sweep_smem(d, true, prec), s>>>(
          bsweep<float>(d, true, c), b->unit_sys, b->bsys, d.r, d.y32);
  }
}

template <int W>
void enq_bwd_w(hbmc_batch *b, const DeviceLayout &d, int prec, int dot, cudaStream_t s) {
  for (int c = d.nc - 1; c >= 0; --c) {
    const unsigned grid = hbmc::nblk(d.tile_ptr[c + 1] - d.tile_ptr[c], (int)per_block(d));
    if (prec == HBMC_PREC_F64)
      hbmc::k_bbwd_w<double, double, W><<<grid, 32 * hbmc::kBWpb, sweep_smem(d, false, prec), s>>>(
          bsweep<double>(d, false, c), b->unit_sys, b->bsys, d.y, d.z, d.r, dot, b->part0);
    else
      hbmc::k_bbwd_w<float, float, W><<<grid, 32 * hbmc::kBWpb, sweep_smem(d, false, prec), s>>>(
          bsweep<float>(d, false, c), b->unit_sys, b->bsys, d.y32, d.z, d.r, dot, b->part0);
  }
}

void enq_fwd(hbmc_batch *b, const View &v, int prec, cudaStream_t s) {
  if (v.d->w == 16) enq_fwd_w<16>(b, *v.d, prec, s);
  else enq_fwd_w<32>(b, *v.d, prec, s);
}

void enq_bwd(hbmc_batch *b, const View &v, int prec, int dot, cudaStream_t s) {
  if (v.d->w == 16) enq_bwd_w<16>(b, *v.d, prec, dot, s);
  else enq_bwd_w<32>(b, *v.d, prec, dot, s);
}

template <int kMode>
void enq_finish(hbmc_batch *b, cudaStream_t s, int use_cond, cudaGraphConditionalHandle h) {
  hbmc::k_bfinish<kMode><<<b->meta.nsys, hbmc::kFinishThreads, 0, s>>>(
      b->meta.nsys, b->meta.nc, b->cu_start, b->cu_count, b->part0, b->part1, b->bsys, b->bg, use_cond, h);
}

template <int W>
void enq_init_w(hbmc_batch *b, const View &v, int prec, cudaStream_t s) {
  const DeviceLayout &d = *v.d;
  const hbmc::ARun a = arun(d);
  const unsigned ug = hbmc::nblk(a.units, (int)per_block(d));
  const size_t sm = (size_t)per_block(d) * a.unit_bytes;
  hbmc::k_bgather_in<<<hbmc::nblk(d.n_pad, 256), 256, 0, s>>>(d.b, d.inv, d.n_pad, b->bg, 0);
  hbmc::k_bgather_in<<<hbmc::nblk(d.n_pad, 256), 256, 0, s>>>(d.x, d.inv, d.n_pad, b->bg, 1);
  hbmc::k_bresid_w<0, W><<<ug, 32 * hbmc::kBWpb, sm, s>>>(a, d.b, d.x, d.r, b->part0, b->part1);
  enq_finish<hbmc::F_INIT>(b, s, 0, 0);
  enq_fwd(b, v, prec, s);
  enq_bwd(b, v, prec, 1, s);
  enq_finish<hbmc::F_RZ_INIT>(b, s, 0, 0);
  hbmc::k_bupdate_p_w<W><<<ug, 32 * hbmc::kBWpb, 0, s>>>(d.bs, a.units, b->unit_sys, b->bsys, d.z, d.p, 0);
}

template <int W>
void enq_body_w(hbmc_batch *b, const View &v, int prec, cudaStream_t s, int use_cond,
                cudaGraphConditionalHandle h) {
  const DeviceLayout &d = *v.d;
  const hbmc::ARun a = arun(d);
  const unsigned ug = hbmc::nblk(a.units, (int)per_block(d));
  const size_t sm = (size_t)per_block(d) * a.unit_bytes;
  hbmc::k_bspmv_w<W><<<ug, 32 * hbmc::kBWpb, sm, s>>>(a, b->unit_sys, b->bsys, d.p, d.q, b->part0);
  enq_finish<hbmc::F_PQ>(b, s, use_cond, h);
  hbmc::k_bupdate_xr_w<W><<<ug, 32 * hbmc::kBWpb, 0, s>>>(d.bs, a.units, b->unit_sys, b->bsys, d.p, d.q, d.x, d.r,
                                                           b->part0);
  enq_finish<hbmc::F_RR>(b, s, use_cond, h);
  enq_fwd(b, v, prec, s);
  enq_bwd(b, v, prec, 1, s);
  enq_finish<hbmc::F_RZ>(b, s, use_cond, h);
  hbmc::k_bupdate_p_w<W><<<ug, 32 * hbmc::kBWpb, 0, s>>>(d.bs, a.units, b->unit_sys, b->bsys, d.z, d.p, 1);
}

template <int W>
void enq_final_w(hbmc_batch *b, const View &v, cudaStream_t s) {
  const DeviceLayout &d = *v.d;
  const hbmc::ARun a = arun(d);
  const unsigned ug = hbmc::nblk(a.units, (int)per_block(d));
  const size_t sm = (size_t)per_block(d) * a.unit_bytes;
  hbmc::k_bgather_out<<<hbmc::nblk(d.n, 256), 256, 0, s>>>(d.x, d.pi, d.n, b->unit_sys, (int64_t)d.bs * d.w,
                                                           b->bsys, b->bg);
  hbmc::k_bresid_w<1, W><<<ug, 32 * hbmc::kBWpb, sm, s>>>(a, d.b, d.x, d.t, b->part0, nullptr);
  enq_finish<hbmc::F_TRUE>(b, s, 0, 0);
}

void enq_init(hbmc_batch *b, const View &v, int prec, cudaStream_t s) {
  if (v.d->w == 16) enq_init_w<16>(b, v, prec, s);
  else enq_init_w<32>(b, v, prec, s);
}

void enq_body(hbmc_batch *b, const View &v, int prec, cudaStream_t s, int use_cond, cudaGraphConditionalHandle h) {
  if (v.d->w == 16) enq_body_w<16>(b, v, prec, s, use_cond, h);
  else enq_body_w<32>(b, v, prec, s, use_cond, h);
}

void enq_final(hbmc_batch *b, const View &v, cudaStream_t s) {
  if (v.d->w == 16) enq_final_w<16>(b, v, s);
  else enq_final_w<32>(b, v, s);
}

hbmc_status build_graph(hbmc_batch *b, const View &v, int prec) {
  cudaGraph_t g = nullptr;
  BCK(cudaGraphCreate(&g, 0));
  b->graph[prec] = g;
  cudaGraphConditionalHandle handle;
  BCK(cudaGraphConditionalHandleCreate(&handle, g, 1, cudaGraphCondAssignDefault));
  cudaStream_t s = b->cap[0], s2 = b->cap[1];
  BCK(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  enq_init(b, v, prec, s);
  cudaStreamCaptureStatus st;
  const cudaGraphNode_t *deps = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, nullptr, &deps, nullptr, &ndeps);
  cudaGraphNode_t loop;
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  if (e == cudaSuccess) {
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    std::vector<cudaGraphNode_t> dv(deps, deps + ndeps);
    e = cudaGraphAddNode(&loop, g, dv.data(), nullptr, dv.size(), &cp);
  }
  if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(s, &loop, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e == cudaSuccess) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(s2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      enq_body(b, v, prec, s2, 1, handle);
      e = cudaStreamEndCapture(s2, &body);
    }
  }
  if (e != cudaSuccess) {
    cudaGraph_t junk;
    cudaStreamEndCapture(s, &junk);
    return berr(b, HBMC_ERR_CUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
  }
  enq_final(b, v, s);
  BCK(cudaStreamEndCapture(s, &g));
  BCK(cudaGetLastError());
  BCK(cudaGraphInstantiate(&b->exec[prec], g, 0));
  return HBMC_OK;
}

const int32_t kBoxes[7][4] = {{1, 1, 1, 1}, {2, 1, 1, 2}, {4, 1, 2, 2}, {8, 2, 2, 2},
                              {16, 2, 2, 4}, {32, 2, 4, 4}, {64, 4, 4, 4}};

bool box_for(int32_t bs, int32_t *box) {
  for (const auto &r : kBoxes)
    if (r[0] == bs) {
      box[0] = r[1];
      box[1] = r[2];
      box[2] = r[3];
      return true;
    }
  return false;
}

std::string fingerprint(int32_t nsys, const hbmc_system *sys) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t v) {
    for (int k = 0; k < 8; ++k) {
      h ^= (v >> (8 * k)) & 0xff;
      h *= 1099511628211ull;
    }
  };
  mix((uint64_t)nsys);
  for (int32_t s = 0; s < nsys; ++s) {
    mix((uint64_t)sys[s].n);
    mix((uint64_t)(sys[s].n ? sys[s].row_ptr[sys[s].n] : 0));
    mix((uint64_t)sys[s].blocking);
  }
  char buf[32];
  std::snprintf(buf, sizeof buf, "%016llx", (unsigned long long)h);
  return buf;
}

template <int W>
void allow_batch(int cap) {
  cudaFuncSetAttribute(hbmc::k_bfwd_w<double, double, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(hbmc::k_bfwd_w<float, float, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(hbmc::k_bbwd_w<double, double, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(hbmc::k_bbwd_w<float, float, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(hbmc::k_bspmv_w<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(hbmc::k_bresid_w<0, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(hbmc::k_bresid_w<1, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
}

}  // namespace

extern "C" {

const char *hbmc_batch_last_error(const hbmc_batch *b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

void hbmc_batch_destroy(hbmc_batch *b) {
  if (!b) return;
  View v;
  if (b->ctx && view(b, v)) {
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(v.dev);
    cudaDeviceSynchronize();
    for (int k = 0; k < 2; ++k) {
      if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
      if (b->graph[k]) cudaGraphDestroy(b->graph[k]);
      if (b->cap[k]) cudaStreamDestroy(b->cap[k]);
    }
    for (void *p : b->allocs) cudaFree(p);
    if (b->h_bsys) cudaFreeHost(b->h_bsys);
    if (b->h_bg) cudaFreeHost(b->h_bg);
    if (prev >= 0) cudaSetDevice(prev);
  }
  hbmc_destroy(b->ctx);
  delete b;
}

hbmc_status hbmc_batch_build(int32_t nsys, const hbmc_system *systems, int32_t bs, const hbmc_options *opt,
                             hbmc_batch **out) {
  return hbmc_batch_build_w(nsys, systems, bs, 32, opt, out);
}

hbmc_status hbmc_batch_build_w(int32_t nsys, const hbmc_system *systems, int32_t bs, int32_t w,
                               const hbmc_options *opt, hbmc_batch **out) {
  if (!out) return berr(nullptr, HBMC_ERR_INVALID_ARG, "out is null");
  if (w != 16 && w != 32) return berr(nullptr, HBMC_ERR_INVALID_ARG, "batch: w must be 16 or 32");
  *out = nullptr;
  hbmc_options o;
  hbmc_default_options(&o);
  if (opt) o = *opt;
  if (o.host_only) return berr(nullptr, HBMC_ERR_INVALID_ARG, "batch: host_only is not supported");
  if (o.nonsymmetric) return berr(nullptr, HBMC_ERR_INVALID_ARG, "batch: only symmetric systems (IC(0), CG)");
  if (o.sell_split) return berr(nullptr, HBMC_ERR_INVALID_ARG, "batch: row splitting is not supported");
  if (o.sell_vslice < 0) return berr(nullptr, HBMC_ERR_INVALID_ARG, "batch: sell_vslice must be >= 0");
  if (o.precision != HBMC_PREC_F64 && o.precision != HBMC_PREC_F32)
    return berr(nullptr, HBMC_ERR_INVALID_ARG, "unknown precision");
  o.sweep_kernel = 0;
  o.sweep_tpb = 0;
  hbmc_batch *b = new hbmc_batch();
  b->precision = o.precision;
  b->loop_mode = o.loop_mode;
  b->check_every = o.check_every > 0 ? o.check_every : 16;
  hbmc::HostLayout g;
  std::string e;
  hbmc_status st;
  try {
    hbmc_options per_sys = o;  // the systems are laid out one by one, the SpMV layout once merged
    per_sys.sell_vslice = 0;
    st = hbmc::build_batch_host(nsys, systems, bs, w, per_sys, g, b->meta, e);
    if (st == HBMC_OK && o.sell_vslice > 0) st = hbmc::plan_vslice(g, o.sell_vslice, e);
  } catch (const std::bad_alloc &) {
    st = HBMC_ERR_OOM;
    e = "host allocation failed";
  }
  if (st == HBMC_OK) st = hbmc::make_ctx_from_layout(std::move(g), o, &b->ctx, e);
  if (st != HBMC_OK) {
    g_batch_err = e;
    delete b;
    return st;
  }
  View v;
  view(b, v);
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(v.dev);
  const hbmc::BatchMeta &m = b->meta;
  const int64_t units = v.d->tile_ptr[v.d->nc];
  auto fail = [&](hbmc_status s) {
    g_batch_err = b->err;
    if (prev >= 0) cudaSetDevice(prev);
    hbmc_batch_destroy(b);
    return s;
  };
  if ((st = bupload(b, b->unit_sys, m.unit_sys)) || (st = bupload(b, b->cu_start, m.cu_start)) ||
      (st = bupload(b, b->cu_count, m.cu_count)) || (st = balloc(b, b->bsys, (size_t)m.nsys)) ||
      (st = balloc(b, b->bg, 1)) || (st = balloc(b, b->part0, (size_t)units)) ||
      (st = balloc(b, b->part1, (size_t)units)) || (st = balloc(b, b->scale, (size_t)m.nsys)) ||
      (st = balloc(b, b->bad, (size_t)m.nsys)))
    return fail(st);
  if (cudaMallocHost(&b->h_bsys, sizeof(BSys) * m.nsys) != cudaSuccess ||
      cudaMallocHost(&b->h_bg, sizeof(BGlob)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap[0], cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap[1], cudaStreamNonBlocking) != cudaSuccess) {
    b->err = "batch: host/stream setup failed";
    return fail(HBMC_ERR_CUDA);
  }
  size_t need = 0;
  for (const hbmc::WarpPlan *wp : {&v.d->wp_f64_f, &v.d->wp_f64_b, &v.d->wp_f32_f, &v.d->wp_f32_b, &v.d->wp_spmv})
    need = std::max(need, (size_t)per_block(*v.d) * wp->warp_bytes);
  if (need > 200 * 1024) {
    b->err = "batch: a level-1 block's same-block run does not fit in shared memory";
    return fail(HBMC_ERR_INVALID_ARG);
  }
  const int cap = 200 * 1024;
  if (w == 16) allow_batch<16>(cap);
  else allow_batch<32>(cap);
  if (cudaGetLastError() != cudaSuccess) {
    b->err = "batch: kernel attribute setup failed";
    return fail(HBMC_ERR_CUDA);
  }
  if (prev >= 0) cudaSetDevice(prev);
  *out = b;
  return HBMC_OK;
}

hbmc_status hbmc_batch_info(const hbmc_batch *bc, int64_t *n_total, int64_t *n_pad_total, int32_t *nc,
                            int64_t *units) {
  hbmc_batch *b = const_cast<hbmc_batch *>(bc);
  if (!b) return berr(nullptr, HBMC_ERR_INVALID_ARG, "null batch");
  View v;
  if (!view(b, v)) return berr(b, HBMC_ERR_INVALID_ARG, "batch has no device context");
  if (n_total) *n_total = v.d->n;
  if (n_pad_total) *n_pad_total = v.d->n_pad;
  if (nc) *nc = v.d->nc;
  if (units) *units = v.d->tile_ptr[v.d->nc];
  return HBMC_OK;
}

hbmc_status hbmc_batch_set_stream(hbmc_batch *b, void *stream) {
  if (!b) return berr(nullptr, HBMC_ERR_INVALID_ARG, "null batch");
  return hbmc_set_stream(b->ctx, stream);
}

hbmc_status hbmc_batch_set_precision(hbmc_batch *b, int32_t precision) {
  if (!b) return berr(nullptr, HBMC_ERR_INVALID_ARG, "null batch");
  if (precision != HBMC_PREC_F64 && precision != HBMC_PREC_F32) return berr(b, HBMC_ERR_INVALID_ARG, "unknown precision");
  b->precision = precision;
  return HBMC_OK;
}

hbmc_status hbmc_batch_ic0(hbmc_batch *b, const double *shifts, int64_t *bad_rows) {
  if (!b) return berr(nullptr, HBMC_ERR_INVALID_ARG, "null batch");
  View v;
  if (!view(b, v)) return berr(b, HBMC_ERR_INVALID_ARG, "batch has no device context");
  const hbmc::BatchMeta &m = b->meta;
  std::vector<double> scale(m.nsys, 1.0);
  for (int32_t s = 0; s < m.nsys; ++s) {
    const double a = shifts ? shifts[s] : 0.0;
    if (!(a > -1.0) || !(a < 1e300)) return berr(b, HBMC_ERR_INVALID_ARG, "shift must be > -1 and finite");
    scale[s] = 1.0 + a;
  }
  b->factored = false;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(v.dev);
  const DeviceLayout &d = *v.d;
  cudaStream_t s = v.s;
  BCK(cudaMemcpyAsync(b->scale, scale.data(), sizeof(double) * m.nsys, cudaMemcpyHostToDevice, s));
  hbmc::k_fill_ll<<<hbmc::nblk(m.nsys, 256), 256, 0, s>>>(b->bad, m.nsys, LLONG_MAX);
  for (int c = 0; c < d.nc; ++c) {
    const int64_t t0 = d.tile_ptr[c], nt = d.tile_ptr[c + 1] - t0;
    hbmc::k_bic0<<<hbmc::nblk(nt * d.w, 128), 128, 0, s>>>(d.lrp, d.lci, d.laval, d.adiag, b->scale,
                                                            b->unit_sys, d.lval, d.ldiag, d.dinv, d.bs, d.w, t0, nt,
                                                            b->bad);
  }
  hbmc::enqueue_scatter_factor(d, true, s);
  std::vector<long long> bad(m.nsys);
  BCK(cudaMemcpyAsync(bad.data(), b->bad, sizeof(long long) * m.nsys, cudaMemcpyDeviceToHost, s));
  BCK(cudaStreamSynchronize(s));
  if (prev >= 0) cudaSetDevice(prev);
  hbmc_status st = HBMC_OK;
  for (int32_t k = 0; k < m.nsys; ++k) {
    int64_t row = -1;
    if (bad[k] != LLONG_MAX) {
      // the failing padded row belongs to system k: back to its own numbering
      const int64_t gi = bad[k];
      row = -2;
      if (gi >= 0 && gi < (int64_t)d.n_pad) {
        std::vector<int32_t> invv(1);
        cudaMemcpy(invv.data(), d.inv + gi, sizeof(int32_t), cudaMemcpyDeviceToHost);
        row = invv[0] >= 0 ? invv[0] - m.orig0[k] : -2;
      }
      st = HBMC_ERR_NOT_SPD_PIVOT;
    }
    if (bad_rows) bad_rows[k] = row;
  }
  b->factored = true;  // systems that failed report it; the rest are usable
  if (st != HBMC_OK) b->err = "IC(0) pivot not positive in at least one system";
  return st;
}

hbmc_status hbmc_batch_iccg(hbmc_batch *b, const double *b_dev, double *x_dev, double tol, int64_t maxit,
                            int64_t *iters, double *relres, double *true_relres, int32_t *status,
                            double *solve_ms) {
  if (!b) return berr(nullptr, HBMC_ERR_INVALID_ARG, "null batch");
  View v;
  if (!view(b, v)) return berr(b, HBMC_ERR_INVALID_ARG, "batch has no device context");
  if (!b->factored) return berr(b, HBMC_ERR_NOT_FACTORED, "hbmc_batch_ic0 has not run");
  if (!(tol > 0.0) || maxit < 0) return berr(b, HBMC_ERR_INVALID_ARG, "tol must be > 0 and maxit >= 0");
  if (!b_dev || !x_dev) return berr(b, HBMC_ERR_INVALID_ARG, "null vector");
  const hbmc::BatchMeta &m = b->meta;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(v.dev);
  cudaStream_t s = v.s;
  const int prec = b->precision;
  BGlob g0;
  std::memset(&g0, 0, sizeof g0);
  g0.tol = tol;
  g0.maxit = maxit;
  g0.active = m.nsys;
  g0.user_b = b_dev;
  g0.user_x = x_dev;
  *b->h_bg = g0;
  BCK(cudaMemcpyAsync(b->bg, b->h_bg, sizeof(BGlob), cudaMemcpyHostToDevice, s));
  BCK(cudaMemsetAsync(b->bsys, 0, sizeof(BSys) * m.nsys, s));
  if (b->loop_mode == HBMC_LOOP_GRAPH) {
    if (!b->exec[prec]) {
      hbmc_status st = build_graph(b, v, prec);
      if (st != HBMC_OK) return st;
    }
    BCK(cudaGraphLaunch(b->exec[prec], s));
  } else {
    enq_init(b, v, prec, s);
    for (;;) {
      for (int k = 0; k < b->check_every; ++k) enq_body(b, v, prec, s, 0, 0);
      BCK(cudaGetLastError());
      BCK(cudaMemcpyAsync(b->h_bg, b->bg, sizeof(BGlob), cudaMemcpyDeviceToHost, s));
      BCK(cudaStreamSynchronize(s));
      if (b->h_bg->active <= 0) break;
    }
    enq_final(b, v, s);
  }
  BCK(cudaGetLastError());
  BCK(cudaMemcpyAsync(b->h_bsys, b->bsys, sizeof(BSys) * m.nsys, cudaMemcpyDeviceToHost, s));
  BCK(cudaMemcpyAsync(b->h_bg, b->bg, sizeof(BGlob), cudaMemcpyDeviceToHost, s));
  BCK(cudaStreamSynchronize(s));
  if (prev >= 0) cudaSetDevice(prev);
  hbmc_status ret = HBMC_OK;
  for (int32_t k = 0; k < m.nsys; ++k) {
    const BSys &y = b->h_bsys[k];
    hbmc_status st = y.status == hbmc::ST_CONVERGED ? HBMC_OK
                     : y.status == hbmc::ST_MAXIT   ? HBMC_NOT_CONVERGED
                     : y.status == hbmc::ST_BREAKDOWN ? HBMC_ERR_BREAKDOWN
                                                      : HBMC_ERR_CUDA;
    if (st != HBMC_OK && ret == HBMC_OK) ret = st;
    if (iters) iters[k] = y.iters;
    if (relres) relres[k] = y.relres;
    if (true_relres) true_relres[k] = y.true_relres;
    if (status) status[k] = st;
    if (solve_ms) solve_ms[k] = y.t_done >= b->h_bg->t0 ? (double)(y.t_done - b->h_bg->t0) * 1e-6 : 0.0;
  }
  if (ret != HBMC_OK) b->err = "at least one system did not converge";
  return ret;
}

hbmc_status hbmc_batch_features(hbmc_batch *b, float *feat) {
  if (!b || !feat) return berr(b, HBMC_ERR_INVALID_ARG, "null argument");
  View v;
  if (!view(b, v)) return berr(b, HBMC_ERR_INVALID_ARG, "batch has no device context");
  if (v.d->w != 32) return berr(b, HBMC_ERR_INVALID_ARG, "batch features need a batch built with w = 32");
  const hbmc::BatchMeta &m = b->meta;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(v.dev);
  int32_t *ncs = nullptr;
  float *fd = nullptr;
  hbmc_status st = HBMC_OK;
  if (cudaMalloc(&ncs, sizeof(int32_t) * m.nsys) != cudaSuccess ||
      cudaMalloc(&fd, sizeof(float) * m.nsys * HBMC_NUM_FEATURES) != cudaSuccess)
    st = HBMC_ERR_OOM;
  if (st == HBMC_OK && cudaMemcpy(ncs, m.nc_sys.data(), sizeof(int32_t) * m.nsys, cudaMemcpyHostToDevice) != cudaSuccess)
    st = HBMC_ERR_CUDA;
  if (st == HBMC_OK) st = hbmc::features_on_device(*v.d, m.nsys, b->cu_start, b->cu_count, ncs, fd, v.s, b->err);
  if (st == HBMC_OK &&
      cudaMemcpy(feat, fd, sizeof(float) * m.nsys * HBMC_NUM_FEATURES, cudaMemcpyDeviceToHost) != cudaSuccess)
    st = HBMC_ERR_CUDA;
  cudaFree(ncs);
  cudaFree(fd);
  if (prev >= 0) cudaSetDevice(prev);
  return st;
}

hbmc_status hbmc_batch_autotune(int32_t nsys, const hbmc_system *systems, const int32_t *bs_candidates,
                                int32_t ncand, const hbmc_options *opt, const double *b_dev, double tol,
                                int64_t maxit, const char *cache_path, int32_t *best_bs, double *ms) {
  const int32_t w32 = 32, v0 = 0;
  int32_t best_w = 0, best_v = 0;
  return hbmc_batch_autotune_w(nsys, systems, bs_candidates, ncand, &w32, 1, &v0, 1, opt, b_dev, tol, maxit,
                               cache_path, best_bs, &best_w, &best_v, ms);
}

hbmc_status hbmc_batch_autotune_w(int32_t nsys, const hbmc_system *systems, const int32_t *bs_candidates,
                                  int32_t nbs, const int32_t *w_candidates, int32_t nw,
                                  const int32_t *vslice_candidates, int32_t nv, const hbmc_options *opt,
                                  const double *b_dev, double tol, int64_t maxit, const char *cache_path,
                                  int32_t *best_bs, int32_t *best_w, int32_t *best_vslice, double *ms) {
  if (!best_bs || !best_w || !best_vslice || !bs_candidates || nbs < 1 || !w_candidates || nw < 1 ||
      !vslice_candidates || nv < 1 || !b_dev)
    return berr(nullptr, HBMC_ERR_INVALID_ARG, "autotune: bad arguments");
  for (int32_t k = 0; k < nw; ++k)
    if (w_candidates[k] != 16 && w_candidates[k] != 32)
      return berr(nullptr, HBMC_ERR_INVALID_ARG, "autotune: w candidates must be 16 or 32");
  for (int32_t k = 0; k < nv; ++k)
    if (vslice_candidates[k] < 0) return berr(nullptr, HBMC_ERR_INVALID_ARG, "autotune: vslice candidates must be >= 0");
  // the cache key covers the candidate sets as well as the systems
  std::string key = fingerprint(nsys, systems);
  for (int32_t k = 0; k < nbs; ++k) key += "b" + std::to_string(bs_candidates[k]);
  for (int32_t k = 0; k < nw; ++k) key += "w" + std::to_string(w_candidates[k]);
  for (int32_t k = 0; k < nv; ++k) key += "v" + std::to_string(vslice_candidates[k]);
  const int32_t ncand = nbs * nw * nv;
  if (cache_path) {
    std::ifstream in(cache_path);
    std::string line;
    while (std::getline(in, line)) {
      std::istringstream ls(line);
      std::string k;
      int32_t vb = 0, vw = 0, vv = 0;
      if ((ls >> k >> vb >> vw >> vv) && k == key) {
        *best_bs = vb;
        *best_w = vw;
        *best_vslice = vv;
        if (ms)
          for (int32_t c = 0; c < ncand; ++c) ms[c] = -1.0;
        return HBMC_OK;
      }
    }
  }
  hbmc_options o;
  hbmc_default_options(&o);
  if (opt) o = *opt;
  double best = 1e300;
  *best_bs = -1;
  *best_w = -1;
  *best_vslice = -1;
  int64_t n_total = 0;
  for (int32_t s = 0; s < nsys; ++s) n_total += systems[s].n;
  double *x = nullptr;
  if (cudaMalloc(&x, sizeof(double) * (n_total ? n_total : 1)) != cudaSuccess)
    return berr(nullptr, HBMC_ERR_OOM, "autotune: no memory for x");
  for (int32_t c = 0; c < ncand; ++c) {
    {
      const int32_t cb = c / (nw * nv), cw = (c / nv) % nw, cv = c % nv;
      if (ms) ms[c] = -1.0;
      const int32_t bs = bs_candidates[cb], w = w_candidates[cw];
      if (!box_for(bs, o.box)) continue;
      o.sell_vslice = vslice_candidates[cv];
      hbmc_batch *b = nullptr;
      if (hbmc_batch_build_w(nsys, systems, bs, w, &o, &b) != HBMC_OK) continue;
      double t = -1.0;
      if (hbmc_batch_ic0(b, nullptr, nullptr) == HBMC_OK) {
        View v;
        view(b, v);
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        bool ok = true;
        for (int rep = 0; rep < 2 && ok; ++rep) {
          cudaMemsetAsync(x, 0, sizeof(double) * n_total, v.s);
          cudaEventRecord(e0, v.s);
          ok = hbmc_batch_iccg(b, b_dev, x, tol, maxit, nullptr, nullptr, nullptr, nullptr, nullptr) == HBMC_OK;
          cudaEventRecord(e1, v.s);
          cudaEventSynchronize(e1);
        }
        float f = 0.f;
        if (ok && cudaEventElapsedTime(&f, e0, e1) == cudaSuccess) t = f;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
      }
      hbmc_batch_destroy(b);
      if (ms) ms[c] = t;
      if (t > 0 && t < best) {
        best = t;
        *best_bs = bs;
        *best_w = w;
        *best_vslice = vslice_candidates[cv];
      }
    }
  }
  cudaFree(x);
  if (*best_bs < 0) return berr(nullptr, HBMC_ERR_INVALID_ARG, "autotune: no candidate solved the batch");
  if (cache_path) {
    std::ofstream outf(cache_path, std::ios::app);
    outf << key << " " << *best_bs << " " << *best_w << " " << *best_vslice << "\n";
  }
  return HBMC_OK;
}

}  // extern "C"

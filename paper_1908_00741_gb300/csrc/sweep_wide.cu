// Substitution sweeps with one CUDA block of NT threads per
// level-1 block, for colors that have few level-1 blocks.
//
// With one warp per level-1 block a color of U level-1 blocks runs U warps;
// when U is near the SM count (matrices with many colors: a 27-point stencil
// in a random order needs over 20) the GPU idles and each warp walks its
// level-1 block's other-color couplings (Eq. "for3") a few entries per lane
// at a time, one dependent trip to memory after another.  Here the whole
// block does that walk at once:
//   1. the level-1 block's record, right-hand side and dinv segments;
//   2. every thread takes a share of the other-color run -- kWideU entries
//      per round, column and coefficient loads first, then the gathers -- and
//      parks coefficient and gathered value in shared memory; the same-block
//      run is staged next to them;
//   3. one thread per row adds its terms in the layout's order (farthest
//      column from the diagonal first) out of shared memory.
//   The other-color run is read from a copy without SELL padding: the
//   level-1 block's rows one after another (a row's entries contiguous, in
//   the same order), so rows of very unequal length -- the imbalance that
//   Section 5.2.2 discusses for SELL -- cost their own entries only.  When
//   the run is too long for shared memory (rows of 80 to 240 entries: a
//   structural matrix), 2 and 3 repeat over groups of consecutive rows, as
//   many as the staging area holds, each row summed in one go.
//   4. lanes j < w run the bs-step chains (Eqs. "y2-2", "y2-3");
//   5. the rows are stored (backward: with the fused r.z).
// The arithmetic and its order are those of every other sweep kernel, so
// the results are bit-identical to them and to the oracle.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <type_traits>

#include "device_util.cuh"
#include "hbmc_internal.h"
#include "kernels.h"
#include "warp_common.cuh"

namespace hbmc {
namespace {

constexpr int kWideU = 8;
constexpr size_t kWideSmemBudget = 200 * 1024;
constexpr uint32_t kWideRecInts = 160;  // record of bs <= 64: 8 + 2 bs ints, rounded
constexpr uint32_t kWideRecOff = 16;    // record after the bulk-copy variant's mbarrier
constexpr uint64_t kWideWaitNs = 4000000000ull;
// Under automatic selection a color uses these kernels when its level-1
// blocks' other-color runs are long -- a warp would walk at least
// kWideMinRun entries, 8 per lane per trip to memory, one trip after
// another -- or when it has fewer than two level-1 blocks per SM.  Measured at
// 128^3 (7-point, runs of 768 entries) the warp kernels win; on the 27-point
// and 3-DOF matrices in a random order (runs of 5000-9000) these do.
constexpr int64_t kWideMinRun = 2048;
// ... and their split form when the unpadded runs average this many entries.
constexpr int64_t kSplitMinRun = 12288;
constexpr int kSplitU = 16;  // split form: entries per thread and trip (256 threads: 4096 a trip)

template <typename T>
struct WideArgs {
  const int32_t *rec;      // per level-1 block records (the same-block run)
  const int64_t *x_ptr;    // unpadded other-color runs: starts
  const int32_t *x_rel;    //   row offsets, x_stride ints per level-1 block
  const int32_t *x_col;
  const T *x_val;
  const uint8_t *i_m;
  const T *i_val;
  const T *dinv;
  int rec_ints, bs, w, lw, chunk, x_stride;
  int gsteps;      // split variant: steps per CUDA block
  unsigned *ucnt;  // split variant: per level-1 block arrival counters (zero between launches)
  int64_t tile0;
  uint32_t off_xr, off_ts, off_tin, off_ds, off_rr, off_oc, off_vv, off_gv, off_iv, off_im;
};

// Phase 3 for rows [r0, r1), whose other-color entries from run position
// e_beg on are staged in vv / gv.
template <int NT, typename T>
__device__ __forceinline__ void wide_osum(const WideArgs<T> &a, unsigned char *smem, int r0, int r1, int e_beg) {
  const int32_t *xr = reinterpret_cast<const int32_t *>(smem + a.off_xr);
  T *ts = reinterpret_cast<T *>(smem + a.off_ts);
  const T *vv = reinterpret_cast<const T *>(smem + a.off_vv) - e_beg;
  const T *gv = reinterpret_cast<const T *>(smem + a.off_gv) - e_beg;
  for (int lr = r0 + (int)threadIdx.x; lr < r1; lr += NT) {
    T acc = ts[lr];
    const int pe = xr[lr + 1];
    for (int p = xr[lr]; p < pe; ++p) acc = fma(-vv[p], gv[p], acc);
    ts[lr] = acc;
  }
}

// The last row r1 > r0 such that rows [r0, r1) fit in `chunk` staged
// entries (xr ascending; the plan makes every single row fit).
__device__ __forceinline__ int rows_fitting(const int32_t *xr, int r0, int R, int chunk) {
  int lo = r0 + 1, hi = R;  // xr[lo] - xr[r0] <= chunk holds
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (xr[mid] - xr[r0] <= chunk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Phases 4-5, common to both ways of staging: the bs-step chains, the stores.
template <int NT, bool FWD, typename T, typename OUT>
__device__ __forceinline__ void wide_chain_store(const WideArgs<T> &a, unsigned char *smem, int64_t row0, OUT *out,
                                                 bool dot, double &rz, float *out32) {
  const int32_t *rs = reinterpret_cast<const int32_t *>(smem + kWideRecOff);
  T *ts = reinterpret_cast<T *>(smem + a.off_ts);
  const T *ds = reinterpret_cast<const T *>(smem + a.off_ds);
  const double *rr = reinterpret_cast<const double *>(smem + a.off_rr);
  const T *iv = reinterpret_cast<const T *>(smem + a.off_iv);
  const uint8_t *im = smem + a.off_im;
  const int tid = threadIdx.x;
  const int R = a.bs << a.lw;
  const int32_t *i_rel = rs + 7 + a.bs;
  // 4.
  if (tid < a.w) {
    const int j = tid;
    for (int q = 0; q < a.bs; ++q) {
      const int l = FWD ? q : a.bs - 1 - q;
      T acc = ts[(l << a.lw) + j];
      const int pe = i_rel[l + 1];
      for (int p = i_rel[l] + j; p < pe; p += a.w) acc = fma(-iv[p], ts[(im[p] << a.lw) + j], acc);
      ts[(l << a.lw) + j] = acc * ds[(l << a.lw) + j];
    }
  }
  __syncthreads();
  // 5.
  for (int lr = tid; lr < R; lr += NT) {
    const T yv = ts[lr];
    out[row0 + lr] = (OUT)yv;
    if constexpr (!FWD && sizeof(T) == 4) out32[row0 + lr] = yv;
    if (!FWD && dot) rz = fma(rr[lr], (double)yv, rz);
  }
}

template <int NT, bool FWD, typename T, typename IN, typename G, typename OUT>
__device__ __forceinline__ void wide_unit(const WideArgs<T> &a, unsigned char *smem, int64_t u, const IN *in,
                                          const G *gsrc, OUT *out, const double *r, bool dot, double &rz,
                                          float *out32 = nullptr) {
  int32_t *rs = reinterpret_cast<int32_t *>(smem + kWideRecOff);
  int32_t *xr = reinterpret_cast<int32_t *>(smem + a.off_xr);
  T *ts = reinterpret_cast<T *>(smem + a.off_ts);
  T *ds = reinterpret_cast<T *>(smem + a.off_ds);
  double *rr = reinterpret_cast<double *>(smem + a.off_rr);
  T *vv = reinterpret_cast<T *>(smem + a.off_vv);
  T *gv = reinterpret_cast<T *>(smem + a.off_gv);
  T *iv = reinterpret_cast<T *>(smem + a.off_iv);
  uint8_t *im = smem + a.off_im;
  const int tid = threadIdx.x;
  const int R = a.bs << a.lw;
  const int64_t row0 = u * (int64_t)R;
  // 1.
  const int32_t *rc = a.rec + u * a.rec_ints;
  for (int k = tid; k < a.rec_ints; k += NT) rs[k] = rc[k];
  const int32_t *xg = a.x_rel + u * a.x_stride;
  for (int k = tid; k <= R; k += NT) xr[k] = xg[k];
  const int64_t xbeg = a.x_ptr[u];
  for (int lr = tid; lr < R; lr += NT) {
    ts[lr] = (T)in[row0 + lr];
    ds[lr] = a.dinv[row0 + lr];
    if (!FWD && dot) rr[lr] = r[row0 + lr];
  }
  __syncthreads();
  const int ilen = rs[1];
  const int64_t ibeg = rec64(rs, 4);
  for (int e = tid; e < ilen; e += NT) {
    iv[e] = a.i_val[ibeg + e];
    im[e] = a.i_m[ibeg + e];
  }
  // 2.-3., over groups of rows [r0, r1) whose entries fit in a.chunk (one
  // group when the whole run does)
  for (int r0 = 0; r0 < R;) {
    const int r1 = rows_fitting(xr, r0, R, a.chunk);
    const int e_beg = xr[r0], e_end = xr[r1];
    for (int e0 = e_beg + tid; e0 < e_end; e0 += NT * kWideU) {
      int32_t c[kWideU];
      T v[kWideU], g[kWideU];
#pragma unroll
      for (int k = 0; k < kWideU; ++k) {
        const int e = e0 + k * NT;
        if (e < e_end) {
          c[k] = a.x_col[xbeg + e];
          v[k] = a.x_val[xbeg + e];
        }
      }
#pragma unroll
      for (int k = 0; k < kWideU; ++k)
        if (e0 + k * NT < e_end) g[k] = (T)gsrc[c[k]];
#pragma unroll
      for (int k = 0; k < kWideU; ++k) {
        const int e = e0 + k * NT;
        if (e < e_end) {
          vv[e - e_beg] = v[k];
          gv[e - e_beg] = g[k];
        }
      }
    }
    __syncthreads();
    wide_osum<NT, T>(a, smem, r0, r1, e_beg);
    __syncthreads();
    r0 = r1;
  }
  wide_chain_store<NT, FWD, T, OUT>(a, smem, row0, out, dot, rz, out32);
}

// The same with w = 32 and every contiguous operand moved by bulk copy
// (cp.async.bulk onto one mbarrier): right-hand side, dinv and r start with
// the record load; the record then gives the runs -- columns and coefficients
// of the other-color run, the same-block run -- and the only loads left to
// the threads are the gathers.  Three dependent trips to memory in all.
// Returns false when the bounded wait ran out (the solve is then stopped).
template <int NT, bool FWD, typename T, typename IN, typename G, typename OUT>
__device__ __forceinline__ bool wide_unit_tma(const WideArgs<T> &a, unsigned char *smem, int64_t u, const IN *in,
                                              const G *gsrc, OUT *out, const double *r, bool dot, double &rz,
                                              Scalars *sc, float *out32 = nullptr) {
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  int32_t *rs = reinterpret_cast<int32_t *>(smem + kWideRecOff);
  int32_t *xr = reinterpret_cast<int32_t *>(smem + a.off_xr);
  T *ts = reinterpret_cast<T *>(smem + a.off_ts);
  IN *tin = reinterpret_cast<IN *>(smem + a.off_tin);  // == ts when IN is T
  T *ds = reinterpret_cast<T *>(smem + a.off_ds);
  double *rr = reinterpret_cast<double *>(smem + a.off_rr);
  int32_t *oc = reinterpret_cast<int32_t *>(smem + a.off_oc);
  T *vv = reinterpret_cast<T *>(smem + a.off_vv);
  T *gv = reinterpret_cast<T *>(smem + a.off_gv);
  T *iv = reinterpret_cast<T *>(smem + a.off_iv);
  uint8_t *im = smem + a.off_im;
  const int tid = threadIdx.x;
  const uint32_t R = (uint32_t)a.bs * 32u;
  const int64_t row0 = u * (int64_t)R;
  const bool want_r = !FWD && dot;
  const uint32_t xbytes = (uint32_t)a.x_stride * 4u;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
    mbar_expect_tx(bar, R * (uint32_t)(sizeof(IN) + sizeof(T)) + (want_r ? R * 8u : 0u) + xbytes);
    tma_load_1d(tin, in + row0, R * (uint32_t)sizeof(IN), bar);
    tma_load_1d(ds, a.dinv + row0, R * (uint32_t)sizeof(T), bar);
    if (want_r) tma_load_1d(rr, r + row0, R * 8u, bar);
    tma_load_1d(xr, a.x_rel + u * a.x_stride, xbytes, bar);
  }
  const int32_t *rc = a.rec + u * a.rec_ints;
  for (int k = tid; k < a.rec_ints; k += NT) rs[k] = rc[k];
  __shared__ int64_t s_x[2];
  if (tid < 2) s_x[tid] = a.x_ptr[u + tid];
  __syncthreads();
  const int ilen = rs[1];
  const int64_t ibeg = rec64(rs, 4), xbeg = s_x[0];
  const uint32_t xlen = (uint32_t)(s_x[1] - s_x[0]);  // a multiple of 32 entries
  if (tid == 0) {
    mbar_arrive_expect_tx(bar, xlen * (uint32_t)(4 + sizeof(T)) + (uint32_t)ilen * (uint32_t)(1 + sizeof(T)));
    if (xlen > 0) {
      tma_load_1d(oc, a.x_col + xbeg, xlen * 4u, bar);
      tma_load_1d(vv, a.x_val + xbeg, xlen * (uint32_t)sizeof(T), bar);
    }
    if (ilen > 0) {
      tma_load_1d(iv, a.i_val + ibeg, (uint32_t)ilen * (uint32_t)sizeof(T), bar);
      tma_load_1d(im, a.i_m + ibeg, (uint32_t)ilen, bar);
    }
  }
  const uint64_t deadline = global_ns() + kWideWaitNs;
  if (!__syncthreads_and(mbar_wait(bar, 0, deadline) ? 1 : 0)) {
    if (tid == 0) {
      sc->timeout = 1;
      sc->done = 1;
      mbar_wait(bar, 0, deadline + kWideWaitNs);  // let the copies land before the block leaves
    }
    __syncthreads();
    return false;
  }
  if constexpr (!std::is_same<IN, T>::value) {
    for (int lr = tid; lr < (int)R; lr += NT) ts[lr] = (T)tin[lr];
  }
  const int olen = xr[R];
  for (int e0 = tid; e0 < olen; e0 += NT * kWideU) {
    T g[kWideU];
#pragma unroll
    for (int k = 0; k < kWideU; ++k)
      if (e0 + k * NT < olen) g[k] = (T)gsrc[oc[e0 + k * NT]];
#pragma unroll
    for (int k = 0; k < kWideU; ++k)
      if (e0 + k * NT < olen) gv[e0 + k * NT] = g[k];
  }
  __syncthreads();
  wide_osum<NT, T>(a, smem, 0, R, 0);
  __syncthreads();
  wide_chain_store<NT, FWD, T, OUT>(a, smem, row0, out, dot, rz, out32);
  return true;
}

template <typename T, typename Y, int NT, bool TMA>
__global__ void __launch_bounds__(NT)
    k_fwd_wide(const WideArgs<T> a, const double *__restrict__ r, Y *y, Scalars *sc, int check_done) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (check_done && sc->done) return;
  double rz = 0.0;
  if constexpr (TMA)
    wide_unit_tma<NT, true, T, double, Y, Y>(a, smem, a.tile0 + blockIdx.x, r, y, y, nullptr, false, rz, sc);
  else
    wide_unit<NT, true, T, double, Y, Y>(a, smem, a.tile0 + blockIdx.x, r, y, y, nullptr, false, rz);
}

template <typename T, typename Y, int NT, bool TMA>
__global__ void __launch_bounds__(NT)
    k_bwd_wide(const WideArgs<T> a, const Y *__restrict__ yin, double *z, float *z32, const double *__restrict__ r,
               Scalars *sc, int check_done, int dot_mode, double *part, int64_t part_off, int last_launch,
               int64_t part_total) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (check_done && sc->done) return;
  double rz = 0.0;
  if constexpr (TMA)
    wide_unit_tma<NT, false, T, Y, T, double>(a, smem, a.tile0 + blockIdx.x, yin, zgather<T>(z, z32), z, r,
                                              dot_mode != 0, rz, sc, z32);
  else
    wide_unit<NT, false, T, Y, T, double>(a, smem, a.tile0 + blockIdx.x, yin, zgather<T>(z, z32), z, r,
                                          dot_mode != 0, rz, z32);
  if (!dot_mode) return;
  rz_partial(rz, sc, dot_mode, part, part_off + blockIdx.x, last_launch, part_total, gridDim.x);
}

// Split variant (colors with few, long level-1 blocks): CUDA block b works
// on level-1 block u = b / G_n, steps [g G, g G + G) with g = b % G_n.  It
// stages and sums the other-color terms of those rows (phases 2-3, every row
// in one go, the same operations as above) and parks the sums in the output
// rows.  The last CUDA block of u to finish (an arrival counter; no block
// waits for another) reads the R sums back and runs the chains and the
// stores (phases 4-5).  So a level-1 block's gathers spread over G_n SMs
// instead of one.  Returns true in the level-1 block's last CUDA block.
template <int NT, bool FWD, typename T, typename IN, typename G, typename OUT>
__device__ __forceinline__ bool wsplit_unit(const WideArgs<T> &a, unsigned char *smem, int64_t u, int g,
                                            const IN *in, const G *gsrc, OUT *out, const double *r, bool dot,
                                            double &rz, float *out32) {
  int32_t *rs = reinterpret_cast<int32_t *>(smem + kWideRecOff);
  int32_t *xr = reinterpret_cast<int32_t *>(smem + a.off_xr);
  T *ts = reinterpret_cast<T *>(smem + a.off_ts);
  T *ds = reinterpret_cast<T *>(smem + a.off_ds);
  double *rr = reinterpret_cast<double *>(smem + a.off_rr);
  T *vv = reinterpret_cast<T *>(smem + a.off_vv);
  T *gv = reinterpret_cast<T *>(smem + a.off_gv);
  T *iv = reinterpret_cast<T *>(smem + a.off_iv);
  uint8_t *im = smem + a.off_im;
  __shared__ unsigned s_arrived;
  const int tid = threadIdx.x;
  const int R = a.bs << a.lw;
  const int64_t row0 = u * (int64_t)R;
  const int q0 = (g * a.gsteps) << a.lw, q1 = min(R, ((g + 1) * a.gsteps) << a.lw), nq = q1 - q0;
  // 1'. this block's rows: offsets (relative to row q0) and right-hand
  // sides; the record too, so that a last block can fetch the same-block run
  // together with the sums
  const int32_t *xg = a.x_rel + u * a.x_stride + q0;
  for (int k = tid; k <= nq; k += NT) xr[k] = xg[k];
  for (int k = tid; k < nq; k += NT) ts[k] = (T)in[row0 + q0 + k];
  const int32_t *rc = a.rec + u * a.rec_ints;
  for (int k = tid; k < a.rec_ints; k += NT) rs[k] = rc[k];
  const int64_t xbeg = a.x_ptr[u];
  __syncthreads();
  // 2'.-3'. as phases 2-3, over groups of this block's rows, kSplitU
  // entries per thread and trip to memory
  for (int k0 = 0; k0 < nq;) {
    const int k1 = rows_fitting(xr, k0, nq, a.chunk);
    const int e_beg = xr[k0], e_end = xr[k1];
    for (int e0 = e_beg + tid; e0 < e_end; e0 += NT * kSplitU) {
      int32_t c[kSplitU];
      T v[kSplitU], gg[kSplitU];
#pragma unroll
      for (int k = 0; k < kSplitU; ++k) {
        const int e = e0 + k * NT;
        if (e < e_end) {
          c[k] = a.x_col[xbeg + e];
          v[k] = a.x_val[xbeg + e];
        }
      }
#pragma unroll
      for (int k = 0; k < kSplitU; ++k)
        if (e0 + k * NT < e_end) gg[k] = (T)gsrc[c[k]];
#pragma unroll
      for (int k = 0; k < kSplitU; ++k) {
        const int e = e0 + k * NT;
        if (e < e_end) {
          vv[e - e_beg] = v[k];
          gv[e - e_beg] = gg[k];
        }
      }
    }
    __syncthreads();
    for (int k = k0 + tid; k < k1; k += NT) {
      T acc = ts[k];
      const int pe = xr[k + 1];
      for (int p = xr[k]; p < pe; ++p) acc = fma(-vv[p - e_beg], gv[p - e_beg], acc);
      ts[k] = acc;
    }
    __syncthreads();
    k0 = k1;
  }
  for (int k = tid; k < nq; k += NT) out[row0 + q0 + k] = (OUT)ts[k];
  __threadfence();
  __syncthreads();
  const int ng = (a.bs + a.gsteps - 1) / a.gsteps;
  if (tid == 0) s_arrived = atomicAdd(&a.ucnt[u], 1u);
  __syncthreads();
  if (s_arrived != (unsigned)(ng - 1)) return false;
  // 1. (the level-1 block's last CUDA block) every row's sum, dinv, r and the
  // same-block run, in one trip to memory
  __threadfence();
  if (tid == 0) a.ucnt[u] = 0;
  const int ilen = rs[1];
  const int64_t ibeg = rec64(rs, 4);
  for (int lr = tid; lr < R; lr += NT) {
    ts[lr] = (T)__ldcg(out + row0 + lr);
    ds[lr] = a.dinv[row0 + lr];
    if (!FWD && dot) rr[lr] = r[row0 + lr];
  }
  for (int e = tid; e < ilen; e += NT) {
    iv[e] = a.i_val[ibeg + e];
    im[e] = a.i_m[ibeg + e];
  }
  __syncthreads();
  wide_chain_store<NT, FWD, T, OUT>(a, smem, row0, out, dot, rz, out32);
  return true;
}

template <typename T, typename Y, int NT>
__global__ void __launch_bounds__(NT, 2)
    k_fwd_wsplit(const WideArgs<T> a, const double *__restrict__ r, Y *y, Scalars *sc, int check_done) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (check_done && sc->done) return;
  const int ng = (a.bs + a.gsteps - 1) / a.gsteps;
  double rz = 0.0;
  wsplit_unit<NT, true, T, double, Y, Y>(a, smem, a.tile0 + blockIdx.x / ng, (int)(blockIdx.x % ng), r, y, y,
                                         nullptr, false, rz, nullptr);
}

template <typename T, typename Y, int NT>
__global__ void __launch_bounds__(NT, 2)
    k_bwd_wsplit(const WideArgs<T> a, const Y *__restrict__ yin, double *z, float *z32,
                 const double *__restrict__ r, Scalars *sc, int check_done, int dot_mode, double *part,
                 int64_t part_off, int last_launch, int64_t part_total) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (check_done && sc->done) return;
  const int ng = (a.bs + a.gsteps - 1) / a.gsteps;
  double rz = 0.0;
  const bool unit_last = wsplit_unit<NT, false, T, Y, T, double>(
      a, smem, a.tile0 + blockIdx.x / ng, (int)(blockIdx.x % ng), yin, zgather<T>(z, z32), z, r, dot_mode != 0,
      rz, z32);
  if (!dot_mode || !unit_last) return;
  // one partial per level-1 block; the launch's last one reduces
  rz_partial(rz, sc, dot_mode, part, part_off + blockIdx.x / ng, last_launch, part_total, gridDim.x / ng);
}

uint32_t a16(uint64_t v) { return (uint32_t)((v + 15) & ~uint64_t(15)); }

// Row offsets of a level-1 block's unpadded run: R + 1 ints, padded to a
// multiple of 4 (16 bytes) so that each block's offsets can be bulk-copied.
int x_stride_of(int bs, int w) { return (bs * w + 1 + 3) / 4 * 4; }

// Shared-memory plan: plain-load staging (tma = false) or bulk-copy staging
// (tma = true, w = 32; adds the column run and, for FP32 forward sweeps, a
// double landing area for r).
WidePlan plan_whole(int bs, int w, bool fwd, bool tma, int rec_ints, int64_t max_o, int64_t max_i, size_t tsize) {
  WidePlan p;
  const uint64_t R = (uint64_t)bs * w;
  p.off_xr = a16((uint64_t)kWideRecOff + (uint64_t)kWideRecInts * 4);
  p.off_ts = a16(p.off_xr + (uint64_t)x_stride_of(bs, w) * 4);
  uint64_t next = p.off_ts + R * tsize;
  p.off_tin = p.off_ts;
  if (tma && fwd && tsize != 8) {
    p.off_tin = a16(next);
    next = p.off_tin + R * 8;
  }
  p.off_ds = a16(next);
  p.off_rr = a16(p.off_ds + R * tsize);
  p.off_oc = a16(p.off_rr + (fwd ? 0 : R * 8));
  p.off_vv = a16(p.off_oc + (tma ? (uint64_t)max_o * 4 : 0));
  p.off_gv = a16(p.off_vv + (uint64_t)max_o * tsize);
  p.off_iv = a16(p.off_gv + (uint64_t)max_o * tsize);
  p.off_im = a16(p.off_iv + (uint64_t)max_i * tsize);
  const uint64_t total = a16(p.off_im + (uint64_t)max_i);
  p.smem_bytes = (uint32_t)std::min<uint64_t>(total, 0xffffffffu);
  p.ok = rec_ints <= (int)kWideRecInts && total <= kWideSmemBudget && (!tma || w == 32);
  p.chunk = (int32_t)std::min<int64_t>(max_o, INT32_MAX);
  return p;
}

// The whole other-color run staged at once when it fits; else (plain loads
// only) as many entries per round as the budget leaves, if that holds the
// longest row (max_step).
WidePlan plan_one(int bs, int w, bool fwd, bool tma, int rec_ints, int64_t max_o, int64_t max_i, int64_t max_step,
                  size_t tsize) {
  WidePlan p = plan_whole(bs, w, fwd, tma, rec_ints, max_o, max_i, tsize);
  if (p.ok || tma || rec_ints > (int)kWideRecInts) return p;
  const WidePlan z = plan_whole(bs, w, fwd, false, rec_ints, 0, max_i, tsize);
  if (z.smem_bytes + 64 >= kWideSmemBudget) return p;
  const int64_t cap = (int64_t)(kWideSmemBudget - z.smem_bytes - 64) / (int64_t)(2 * tsize) / 32 * 32;
  if (cap < max_step || cap < 32) return p;
  p = plan_whole(bs, w, fwd, false, rec_ints, cap, max_i, tsize);
  p.chunk = (int32_t)cap;
  return p;
}

// Split form: one step per CUDA block, a staging area for about three CUDA
// blocks per SM (more if the longest row needs it).
constexpr size_t kSplitSmem = 72 * 1024;
WidePlan plan_split_form(int bs, int w, bool fwd, int rec_ints, int64_t max_i, int64_t max_row, size_t tsize) {
  WidePlan p;
  const WidePlan z = plan_whole(bs, w, fwd, false, rec_ints, 0, max_i, tsize);
  if (!z.ok || rec_ints > (int)kWideRecInts) return p;
  for (size_t budget = kSplitSmem; budget <= kWideSmemBudget; budget += 32 * 1024) {
    if (z.smem_bytes + 64 >= budget) continue;
    const int64_t cap = (int64_t)(budget - z.smem_bytes - 64) / (int64_t)(2 * tsize) / 32 * 32;
    if (cap < max_row || cap < 32) continue;
    p = plan_whole(bs, w, fwd, false, rec_ints, cap, max_i, tsize);
    p.chunk = (int32_t)cap;
    return p;
  }
  return p;
}

const WidePlan &split_plan(const DeviceLayout &d, bool fwd, int prec) {
  return prec == HBMC_PREC_F64 ? (fwd ? d.ws_f64_f : d.ws_f64_b) : (fwd ? d.ws_f32_f : d.ws_f32_b);
}

const WidePlan &wide_plan(const DeviceLayout &d, bool fwd, int prec) {
  return prec == HBMC_PREC_F64 ? (fwd ? d.wd_f64_f : d.wd_f64_b) : (fwd ? d.wd_f32_f : d.wd_f32_b);
}

const WidePlan &wide_tma_plan(const DeviceLayout &d, bool fwd, int prec) {
  return prec == HBMC_PREC_F64 ? (fwd ? d.wt_f64_f : d.wt_f64_b) : (fwd ? d.wt_f32_f : d.wt_f32_b);
}

template <typename T>
WideArgs<T> wide_args(const DeviceLayout &d, bool fwd, int c, const WidePlan &p) {
  WideArgs<T> a;
  a.rec = fwd ? d.rec_f : d.rec_b;
  a.rec_ints = d.rec_ints;
  a.x_ptr = fwd ? d.fx_ptr : d.bx_ptr;
  a.x_rel = fwd ? d.fx_rel : d.bx_rel;
  a.x_col = fwd ? d.fx_col : d.bx_col;
  a.x_stride = x_stride_of(d.bs, d.w);
  a.i_m = fwd ? d.fi_m : d.bi_m;
  if constexpr (sizeof(T) == 8) {
    a.x_val = (const T *)(fwd ? d.fx_val : d.bx_val);
    a.i_val = (const T *)(fwd ? d.fi_val : d.bi_val);
    a.dinv = (const T *)(fwd ? d.dinv : d.dinvb);
  } else {
    a.x_val = (const T *)(fwd ? d.fx_val32 : d.bx_val32);
    a.i_val = (const T *)(fwd ? d.fi_val32 : d.bi_val32);
    a.dinv = (const T *)(fwd ? d.dinv32 : d.dinvb32);
  }
  a.bs = d.bs;
  a.w = d.w;
  a.lw = d.lw;
  a.tile0 = d.tile_ptr[c];
  a.chunk = p.chunk;
  a.gsteps = 1;
  a.ucnt = d.ucnt;
  a.off_xr = p.off_xr;
  a.off_ts = p.off_ts;
  a.off_tin = p.off_tin;
  a.off_ds = p.off_ds;
  a.off_rr = p.off_rr;
  a.off_oc = p.off_oc;
  a.off_vv = p.off_vv;
  a.off_gv = p.off_gv;
  a.off_iv = p.off_iv;
  a.off_im = p.off_im;
  return a;
}

template <typename K>
cudaError_t allow(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWideSmemBudget);
}

}  // namespace

void plan_wide_kernels(const HostLayout &h, DeviceLayout &d) {
  // Layouts without the unpadded runs (the batched solver's merged layout)
  // leave every plan unusable and every color on the warp kernels.
  const size_t nx = (size_t)h.ntiles + 1;
  if (h.fx_ptr.size() != nx || h.bx_ptr.size() != nx || h.rec_f.empty() || h.rec_b.empty() || !d.fx_ptr ||
      !d.bx_ptr || !d.ucnt) {
    d.wide_f.assign(h.nc, 0);
    d.wide_b.assign(h.nc, 0);
    return;
  }
  for (int dir = 0; dir < 2; ++dir) {
    const std::vector<int32_t> &rec = dir == 0 ? h.rec_f : h.rec_b;
    std::vector<uint8_t> &pick = dir == 0 ? d.wide_f : d.wide_b;
    pick.assign(h.nc, 0);
    for (int c = 0; c < h.nc; ++c) {
      const int64_t u0 = h.tile_ptr[c], u1 = h.tile_ptr[c + 1];
      int64_t run = 0;
      for (int64_t u = u0; u < u1; ++u) run += rec[(size_t)u * h.rec_ints];
      const bool long_runs = u1 > u0 && run >= kWideMinRun * (u1 - u0);
      pick[c] = (long_runs || u1 - u0 < 2 * (int64_t)d.sm_count) ? 1 : 0;
      // fewer level-1 blocks than two per SM, with very long runs (rows of
      // 80 or more entries): spread each level-1 block's gathers over bs
      // CUDA blocks.  Measured: it wins on the structural matrix (runs of
      // 12k-22k entries), loses on the 27-point and 3-DOF ones (5k-9k).
      const std::vector<int64_t> &xp = dir == 0 ? h.fx_ptr : h.bx_ptr;
      const bool very_long = u1 > u0 && xp[u1] - xp[u0] >= kSplitMinRun * (u1 - u0);
      if (pick[c] && very_long && u1 - u0 < 2 * (int64_t)d.sm_count) pick[c] = 2;
    }
  }
  d.ws_f64_f = plan_split_form(h.bs, h.w, true, h.rec_ints, h.max_i_f, h.max_xrow_f, 8);
  d.ws_f64_b = plan_split_form(h.bs, h.w, false, h.rec_ints, h.max_i_b, h.max_xrow_b, 8);
  d.ws_f32_f = plan_split_form(h.bs, h.w, true, h.rec_ints, h.max_i_f, h.max_xrow_f, 4);
  d.ws_f32_b = plan_split_form(h.bs, h.w, false, h.rec_ints, h.max_i_b, h.max_xrow_b, 4);
  // unpadded runs: the longest level-1 block run and the longest row
  for (int tma = 0; tma < 2; ++tma) {
    (tma ? d.wt_f64_f : d.wd_f64_f) = plan_one(h.bs, h.w, true, tma, h.rec_ints, h.max_x_f, h.max_i_f, h.max_xrow_f, 8);
    (tma ? d.wt_f64_b : d.wd_f64_b) = plan_one(h.bs, h.w, false, tma, h.rec_ints, h.max_x_b, h.max_i_b, h.max_xrow_b, 8);
    (tma ? d.wt_f32_f : d.wd_f32_f) = plan_one(h.bs, h.w, true, tma, h.rec_ints, h.max_x_f, h.max_i_f, h.max_xrow_f, 4);
    (tma ? d.wt_f32_b : d.wd_f32_b) = plan_one(h.bs, h.w, false, tma, h.rec_ints, h.max_x_b, h.max_i_b, h.max_xrow_b, 4);
  }
}

template <int NT, bool TMA>
cudaError_t allow_nt() {
  cudaError_t e;
  if ((e = allow(k_fwd_wide<double, double, NT, TMA>)) || (e = allow(k_fwd_wide<float, float, NT, TMA>)) ||
      (e = allow(k_bwd_wide<double, double, NT, TMA>)) || (e = allow(k_bwd_wide<float, float, NT, TMA>)))
    return e;
  return cudaSuccess;
}

constexpr int kSplitThreads = 256;

cudaError_t setup_wide_kernels() {
  cudaError_t e;
  if ((e = allow_nt<256, false>()) || (e = allow_nt<512, false>()) || (e = allow_nt<1024, false>()) ||
      (e = allow_nt<256, true>()) || (e = allow_nt<512, true>()) || (e = allow_nt<1024, true>()))
    return e;
  if ((e = allow(k_fwd_wsplit<double, double, kSplitThreads>)) ||
      (e = allow(k_fwd_wsplit<float, float, kSplitThreads>)) ||
      (e = allow(k_bwd_wsplit<double, double, kSplitThreads>)) ||
      (e = allow(k_bwd_wsplit<float, float, kSplitThreads>)))
    return e;
  return cudaSuccess;
}

bool wide_all(const DeviceLayout &d) { return d.sweep_kernel == 4 || d.sweep_kernel == 6 || d.sweep_kernel == 7; }

// The split form for color c: always under sweep_kernel 7, by the per-color
// pick under automatic selection; it needs its plan and the counters.
static bool use_split(const DeviceLayout &d, bool fwd, int prec, int c) {
  if (!d.ucnt || !split_plan(d, fwd, prec).ok) return false;
  if (d.sweep_kernel == 7) return true;
  if (d.sweep_kernel != 0) return false;
  const std::vector<uint8_t> &v = fwd ? d.wide_f : d.wide_b;
  return c < (int)v.size() && v[c] == 2;
}

bool wide_usable(const DeviceLayout &d, bool fwd, int prec) {
  return (d.sweep_kernel == 0 || wide_all(d)) && d.rec_f && wide_plan(d, fwd, prec).ok;
}

bool wide_preferred(const DeviceLayout &d, bool fwd, int c) {
  if (wide_all(d)) return true;
  if (d.sweep_kernel != 0) return false;
  const std::vector<uint8_t> &v = fwd ? d.wide_f : d.wide_b;
  return c < (int)v.size() && v[c] != 0;
}

unsigned wide_color_grid(const DeviceLayout &d, int c) { return (unsigned)(d.tile_ptr[c + 1] - d.tile_ptr[c]); }

// Threads per level-1 block: all 1024 when the color has about one level-1
// block per SM, fewer when several share an SM.
static int wide_threads(const DeviceLayout &d, int c) {
  const int64_t per_sm = (wide_color_grid(d, c) + d.sm_count - 1) / d.sm_count;
  return per_sm <= 1 ? 1024 : per_sm <= 2 ? 512 : 256;
}

template <typename T, typename Y, int NT, bool TMA>
void fwd_nt(const DeviceLayout &d, int c, const double *r, Y *y, bool check_done, cudaStream_t s, const WidePlan &p) {
  k_fwd_wide<T, Y, NT, TMA><<<wide_color_grid(d, c), NT, p.smem_bytes, s>>>(wide_args<T>(d, true, c, p), r, y, d.sc,
                                                                             check_done ? 1 : 0);
}

template <typename T, typename Y, int NT, bool TMA>
void bwd_nt(const DeviceLayout &d, int c, const Y *yin, const double *r, int dot_mode, bool check_done,
            int64_t part_off, bool last, int64_t part_total, cudaStream_t s, const WidePlan &p) {
  k_bwd_wide<T, Y, NT, TMA><<<wide_color_grid(d, c), NT, p.smem_bytes, s>>>(
      wide_args<T>(d, false, c, p), yin, d.z, d.z32, r, d.sc, check_done ? 1 : 0, dot_mode, d.part, part_off,
      last ? 1 : 0, part_total);
}

template <typename T, typename Y, bool TMA>
void fwd_any(const DeviceLayout &d, int c, const double *r, Y *y, bool check_done, cudaStream_t s,
             const WidePlan &p) {
  switch (wide_threads(d, c)) {
    case 1024: fwd_nt<T, Y, 1024, TMA>(d, c, r, y, check_done, s, p); break;
    case 512: fwd_nt<T, Y, 512, TMA>(d, c, r, y, check_done, s, p); break;
    default: fwd_nt<T, Y, 256, TMA>(d, c, r, y, check_done, s, p); break;
  }
}

template <typename T, typename Y, bool TMA>
void bwd_any(const DeviceLayout &d, int c, const Y *yin, const double *r, int dot_mode, bool check_done,
             int64_t part_off, bool last, int64_t part_total, cudaStream_t s, const WidePlan &p) {
  switch (wide_threads(d, c)) {
    case 1024: bwd_nt<T, Y, 1024, TMA>(d, c, yin, r, dot_mode, check_done, part_off, last, part_total, s, p); break;
    case 512: bwd_nt<T, Y, 512, TMA>(d, c, yin, r, dot_mode, check_done, part_off, last, part_total, s, p); break;
    default: bwd_nt<T, Y, 256, TMA>(d, c, yin, r, dot_mode, check_done, part_off, last, part_total, s, p); break;
  }
}

// Waves of CUDA blocks a color needs with a plan: level-1 blocks per SM over
// the blocks an SM holds (by threads and by shared memory).
static int64_t wide_waves(const DeviceLayout &d, int c, const WidePlan &p) {
  const int64_t per_sm = (wide_color_grid(d, c) + d.sm_count - 1) / d.sm_count;
  const int64_t by_threads = 2048 / wide_threads(d, c);
  const int64_t by_smem = std::max<int64_t>(1, (int64_t)(227 * 1024) / ((int64_t)p.smem_bytes + 1024));
  return (per_sm + std::min(by_threads, by_smem) - 1) / std::min(by_threads, by_smem);
}

// Bulk-copy staging saves trips to memory but holds the column run in shared
// memory too, so fewer CUDA blocks share an SM.  Measured: it wins when a
// color has at most two level-1 blocks per SM (27-point 96^3), loses with
// five (3-DOF 100^3).  So: bulk copies when they need fewer waves, or as
// many and the color has at most two level-1 blocks per SM.
static bool wide_use_tma(const DeviceLayout &d, bool fwd, int prec, int c) {
  const WidePlan &pt = wide_tma_plan(d, fwd, prec);
  if (!pt.ok || d.sweep_kernel == 6) return false;
  const int64_t wt = wide_waves(d, c, pt), wp = wide_waves(d, c, wide_plan(d, fwd, prec));
  return wt < wp || (wt == wp && wide_color_grid(d, c) <= 2 * (int64_t)d.sm_count);
}

void launch_fwd_wide_color(const DeviceLayout &d, int prec, int c, const double *r, bool check_done,
                           cudaStream_t s) {
  if (wide_color_grid(d, c) == 0) return;
  if (use_split(d, true, prec, c)) {
    const WidePlan &p = split_plan(d, true, prec);
    const unsigned grid = wide_color_grid(d, c) * (unsigned)d.bs;
    if (prec == HBMC_PREC_F64)
      k_fwd_wsplit<double, double, kSplitThreads><<<grid, kSplitThreads, p.smem_bytes, s>>>(
          wide_args<double>(d, true, c, p), r, d.y, d.sc, check_done ? 1 : 0);
    else
      k_fwd_wsplit<float, float, kSplitThreads><<<grid, kSplitThreads, p.smem_bytes, s>>>(
          wide_args<float>(d, true, c, p), r, d.y32, d.sc, check_done ? 1 : 0);
    return;
  }
  const WidePlan &pt = wide_tma_plan(d, true, prec);
  const bool tma = wide_use_tma(d, true, prec, c);
  const WidePlan &p = tma ? pt : wide_plan(d, true, prec);
  if (prec == HBMC_PREC_F64) {
    if (tma) fwd_any<double, double, true>(d, c, r, d.y, check_done, s, p);
    else fwd_any<double, double, false>(d, c, r, d.y, check_done, s, p);
  } else {
    if (tma) fwd_any<float, float, true>(d, c, r, d.y32, check_done, s, p);
    else fwd_any<float, float, false>(d, c, r, d.y32, check_done, s, p);
  }
}

void launch_bwd_wide_color(const DeviceLayout &d, int prec, int c, const double *r, int dot_mode, bool check_done,
                           int64_t part_off, bool last, int64_t part_total, cudaStream_t s) {
  if (wide_color_grid(d, c) == 0) return;
  if (use_split(d, false, prec, c)) {
    const WidePlan &p = split_plan(d, false, prec);
    const unsigned grid = wide_color_grid(d, c) * (unsigned)d.bs;
    if (prec == HBMC_PREC_F64)
      k_bwd_wsplit<double, double, kSplitThreads><<<grid, kSplitThreads, p.smem_bytes, s>>>(
          wide_args<double>(d, false, c, p), d.y, d.z, d.z32, r, d.sc, check_done ? 1 : 0, dot_mode, d.part,
          part_off, last ? 1 : 0, part_total);
    else
      k_bwd_wsplit<float, float, kSplitThreads><<<grid, kSplitThreads, p.smem_bytes, s>>>(
          wide_args<float>(d, false, c, p), d.y32, d.z, d.z32, r, d.sc, check_done ? 1 : 0, dot_mode, d.part,
          part_off, last ? 1 : 0, part_total);
    return;
  }
  const WidePlan &pt = wide_tma_plan(d, false, prec);
  const bool tma = wide_use_tma(d, false, prec, c);
  const WidePlan &p = tma ? pt : wide_plan(d, false, prec);
  if (prec == HBMC_PREC_F64) {
    if (tma) bwd_any<double, double, true>(d, c, d.y, r, dot_mode, check_done, part_off, last, part_total, s, p);
    else bwd_any<double, double, false>(d, c, d.y, r, dot_mode, check_done, part_off, last, part_total, s, p);
  } else {
    if (tma) bwd_any<float, float, true>(d, c, d.y32, r, dot_mode, check_done, part_off, last, part_total, s, p);
    else bwd_any<float, float, false>(d, c, d.y32, r, dot_mode, check_done, part_off, last, part_total, s, p);
  }
}

}  // namespace hbmc

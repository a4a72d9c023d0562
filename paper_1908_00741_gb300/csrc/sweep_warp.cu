// Warp-per-unit kernels (w = 32): one warp owns one level-1 block ("unit").
//
// Forward substitution of one color (Eqs. "for2", "for3"): lane j of the
// warp owns BMC block j of the unit and its bs rows (one per step).  Every
// operand of the unit that lies contiguously in memory -- its record of
// slice offsets, the right-hand side and dinv segments and its same-block
// coefficient run -- is read with coalesced loads into the warp's slice of
// shared memory; the couplings to other colors (Eq. "for3") are gathered in
// batches of kChunk independent loads per lane; then each lane runs its own
// bs-step chain (Eqs. "y2-2", "y2-3") without any block-level barrier, so an
// SM runs as many chains at once as it holds warps.  The chains are serial
// and, in FP64 on this GPU, long; running tens of them per SM side by side
// is what hides that.
//
// The same unit walk gives the backward substitution (steps bs..1, fused
// r.z) and SpMV (q = A p over the unit's rows, fused p.q).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "device_util.cuh"
#include "warp_common.cuh"
#include "hbmc_internal.h"
#include "kernels.h"

namespace hbmc {
namespace {

constexpr int kMaxWpb = 4;
constexpr size_t kWarpSmemBudget = 200 * 1024;

template <typename T>
struct WArgs {
  const int32_t *rec;
  const int32_t *o_col;
  const T *o_val;
  const uint8_t *i_m;
  const T *i_val;
  const T *dinv;
  int bs, rec_ints;
  int64_t tile0, ntiles;
  uint32_t off_t, off_d, off_iv, off_im, warp_bytes;
};

template <typename T>
struct WarpSmem {
  int32_t *rs;
  T *ts, *ds, *iv;
  uint8_t *im;
};

template <typename T>
__device__ __forceinline__ WarpSmem<T> warp_smem(unsigned char *smem, const WArgs<T> &a, int warp) {
  unsigned char *ws = smem + (size_t)warp * a.warp_bytes;
  WarpSmem<T> m;
  m.rs = reinterpret_cast<int32_t *>(ws);
  m.ts = reinterpret_cast<T *>(ws + a.off_t);
  m.ds = reinterpret_cast<T *>(ws + a.off_d);
  m.iv = reinterpret_cast<T *>(ws + a.off_iv);
  m.im = ws + a.off_im;
  return m;
}

// Record, per-row segments and the same-block run into the warp's shared memory.
template <typename T, typename IN>
__device__ __forceinline__ void stage_unit(const WArgs<T> &a, const WarpSmem<T> &m, int64_t u,
                                           const IN *in, int lane) {
  const int32_t *rc = a.rec + u * a.rec_ints;
  for (int k = lane; k < a.rec_ints; k += 32) m.rs[k] = rc[k];
  const int64_t row0 = u * (int64_t)a.bs * 32;
#pragma unroll 4
  for (int l = 0; l < a.bs; ++l) {
    const int64_t row = row0 + (l << 5) + lane;
    m.ts[(l << 5) + lane] = (T)in[row];
    m.ds[(l << 5) + lane] = a.dinv[row];
  }
  __syncwarp();
  const int ilen = m.rs[1];
  const int64_t ibeg = rec64(m.rs, 4);
#pragma unroll 4
  for (int e = lane; e < ilen; e += 32) {
    m.iv[e] = a.i_val[ibeg + e];
    m.im[e] = a.i_m[ibeg + e];
  }
}

template <typename T, typename Y>
__global__ void __launch_bounds__(32 * kMaxWpb)
    k_fwd_w(const WArgs<T> a, const double *__restrict__ r, Y *y, const Scalars *sc, int check_done) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (check_done && sc->done) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t u = a.tile0 + (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (u >= a.tile0 + a.ntiles) return;
  const WarpSmem<T> m = warp_smem(smem, a, warp);
  stage_unit<T, double>(a, m, u, r, lane);
  const int32_t *rs = m.rs;
  run_accumulate<T, Y, true>(a.o_col, a.o_val, y, rec64(rs, 2), rs[0], rs + 6, m.ts, lane);
  const int32_t *i_rel = rs + 7 + a.bs;
  for (int l = 0; l < a.bs; ++l) {
    T acc = m.ts[(l << 5) + lane];
    const int pe = i_rel[l + 1];
    for (int p = i_rel[l] + lane; p < pe; p += 32) acc = fma(-m.iv[p], m.ts[(m.im[p] << 5) + lane], acc);
    m.ts[(l << 5) + lane] = acc * m.ds[(l << 5) + lane];
  }
  Y *yo = y + u * (int64_t)a.bs * 32;
#pragma unroll 4
  for (int l = 0; l < a.bs; ++l) yo[(l << 5) + lane] = (Y)m.ts[(l << 5) + lane];
}

template <typename T, typename Y>
__global__ void __launch_bounds__(32 * kMaxWpb)
    k_bwd_w(const WArgs<T> a, const Y *__restrict__ yin, double *z, float *z32, const double *__restrict__ r,
            Scalars *sc, int check_done, int dot_mode, double *part, int64_t part_off, int last_launch,
            int64_t part_total) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (check_done && sc->done) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t u = a.tile0 + (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  double rz = 0.0;
  if (u < a.tile0 + a.ntiles) {
    const WarpSmem<T> m = warp_smem(smem, a, warp);
    stage_unit<T, Y>(a, m, u, yin, lane);
    const int32_t *rs = m.rs;
    run_accumulate<T, T, true>(a.o_col, a.o_val, zgather<T>(z, z32), rec64(rs, 2), rs[0], rs + 6, m.ts, lane);
    const int32_t *i_rel = rs + 7 + a.bs;
    for (int l = a.bs - 1; l >= 0; --l) {
      T acc = m.ts[(l << 5) + lane];
      const int pe = i_rel[l + 1];
      for (int p = i_rel[l] + lane; p < pe; p += 32) acc = fma(-m.iv[p], m.ts[(m.im[p] << 5) + lane], acc);
      m.ts[(l << 5) + lane] = acc * m.ds[(l << 5) + lane];
    }
    const int64_t row0 = u * (int64_t)a.bs * 32;
#pragma unroll 4
    for (int l = 0; l < a.bs; ++l) {
      const double zv = (double)m.ts[(l << 5) + lane];
      z[row0 + (l << 5) + lane] = zv;
      if constexpr (sizeof(T) == 4) z32[row0 + (l << 5) + lane] = m.ts[(l << 5) + lane];
      if (dot_mode) rz = fma(r[row0 + (l << 5) + lane], zv, rz);
    }
  }
  if (!dot_mode) return;
  rz_partial(rz, sc, dot_mode, part, part_off + blockIdx.x, last_launch, part_total, gridDim.x);
}

// q = A p over every unit (all colors in one launch), with p.q and alpha.
template <bool kDot>
__global__ void __launch_bounds__(32 * kMaxWpb)
    k_spmv_w(const int32_t *__restrict__ rec, int rec_ints, const int32_t *__restrict__ a_col,
             const double *__restrict__ a_val, int bs, int64_t ntiles, uint32_t off_t, uint32_t warp_bytes,
             const double *p, double *q, double *part, Scalars *sc) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (kDot && sc->done) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t u = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  double pq = 0.0;
  if (u < ntiles) {
    unsigned char *ws = smem + (size_t)warp * warp_bytes;
    int32_t *rs = reinterpret_cast<int32_t *>(ws);
    double *ts = reinterpret_cast<double *>(ws + off_t);
    const int32_t *rc = rec + u * rec_ints;
    for (int k = lane; k < rec_ints; k += 32) rs[k] = rc[k];
    for (int l = 0; l < bs; ++l) ts[(l << 5) + lane] = 0.0;
    __syncwarp();
    run_accumulate<double, double, false>(a_col, a_val, p, rec64(rs, 2), rs[0], rs + 6, ts, lane);
    const int64_t row0 = u * (int64_t)bs * 32;
#pragma unroll 4
    for (int l = 0; l < bs; ++l) {
      const double qv = ts[(l << 5) + lane];
      q[row0 + (l << 5) + lane] = qv;
      if (kDot) pq = fma(p[row0 + (l << 5) + lane], qv, pq);
    }
  }
  if (!kDot) return;
  const double v = block_sum_rt(pq);
  if (!publish(part + blockIdx.x, &v, 1, &sc->cnt[CNT_PQ], gridDim.x)) return;
  __threadfence();
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < gridDim.x; k += blockDim.x) acc += __ldcg(part + k);
  const double s = block_sum_rt(acc);
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

uint32_t al16(uint64_t v) { return (uint32_t)((v + 15) & ~uint64_t(15)); }

WarpPlan plan_warp(int bs, int lanes, int rec_ints, int64_t max_i, size_t tsize) {
  WarpPlan w;
  const uint64_t R = (uint64_t)bs * lanes;
  w.off_t = al16((uint64_t)rec_ints * 4);
  w.off_d = al16(w.off_t + R * tsize);
  w.off_iv = al16(w.off_d + R * tsize);
  w.off_im = al16(w.off_iv + (uint64_t)max_i * tsize);
  w.warp_bytes = al16(w.off_im + (uint64_t)max_i);
  w.wpb = 0;
  for (int k = kMaxWpb; k >= 1; k >>= 1)
    if ((uint64_t)k * w.warp_bytes <= kWarpSmemBudget) {
      w.wpb = k;
      break;
    }
  return w;
}

template <typename T>
WArgs<T> warp_args(const DeviceLayout &d, bool fwd, int c, const WarpPlan &w) {
  WArgs<T> a;
  a.rec = fwd ? d.rec_f : d.rec_b;
  a.rec_ints = d.rec_ints;
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
  a.tile0 = d.tile_ptr[c];
  a.ntiles = d.tile_ptr[c + 1] - d.tile_ptr[c];
  a.off_t = w.off_t;
  a.off_d = w.off_d;
  a.off_iv = w.off_iv;
  a.off_im = w.off_im;
  a.warp_bytes = w.warp_bytes;
  return a;
}

unsigned warp_grid(int64_t units, int wpb) { return (unsigned)((units + wpb - 1) / wpb); }

const WarpPlan &plan_of(const DeviceLayout &d, bool fwd, int prec) {
  return prec == HBMC_PREC_F64 ? (fwd ? d.wp_f64_f : d.wp_f64_b) : (fwd ? d.wp_f32_f : d.wp_f32_b);
}

}  // namespace

void plan_warp_kernels(const HostLayout &h, DeviceLayout &d) {
  // sized for one level-1 block of bs * w rows (the batched solver's
  // kernels also run w = 16, two level-1 blocks per warp)
  const int lanes = h.w == 16 ? 16 : 32;
  d.wp_f64_f = plan_warp(h.bs, lanes, h.rec_ints, h.max_i_f, 8);
  d.wp_f64_b = plan_warp(h.bs, lanes, h.rec_ints, h.max_i_b, 8);
  d.wp_f32_f = plan_warp(h.bs, lanes, h.rec_ints, h.max_i_f, 4);
  d.wp_f32_b = plan_warp(h.bs, lanes, h.rec_ints, h.max_i_b, 4);
  WarpPlan s;
  s.off_t = al16((uint64_t)h.rec_ints * 4);
  s.warp_bytes = al16(s.off_t + (uint64_t)h.bs * lanes * 8);
  s.wpb = (uint64_t)kMaxWpb * s.warp_bytes <= kWarpSmemBudget ? kMaxWpb : 1;
  d.wp_spmv = s;
}

cudaError_t setup_warp_kernels() {
  cudaError_t e;
  const int cap = (int)kWarpSmemBudget;
  if ((e = cudaFuncSetAttribute(k_fwd_w<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap))) return e;
  if ((e = cudaFuncSetAttribute(k_fwd_w<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap))) return e;
  if ((e = cudaFuncSetAttribute(k_bwd_w<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap))) return e;
  if ((e = cudaFuncSetAttribute(k_bwd_w<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap))) return e;
  if ((e = cudaFuncSetAttribute(k_spmv_w<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap))) return e;
  if ((e = cudaFuncSetAttribute(k_spmv_w<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap))) return e;
  return cudaSuccess;
}

bool warp_usable(const DeviceLayout &d, bool fwd, int prec) {
  return (d.sweep_kernel == 0 || d.sweep_kernel == 3) && d.w == 32 && d.rec_f && plan_of(d, fwd, prec).wpb > 0;
}

bool warp_spmv_usable(const DeviceLayout &d) { return d.sweep_kernel == 3 && d.w == 32 && d.rec_a && d.wp_spmv.wpb > 0; }

int64_t warp_partials_needed(const DeviceLayout &d) {
  int64_t need = 0;
  for (const WarpPlan *w : {&d.wp_f64_b, &d.wp_f32_b}) {
    if (w->wpb <= 0) continue;
    int64_t t = 0;
    for (int c = 0; c < d.nc; ++c) t += warp_grid(d.tile_ptr[c + 1] - d.tile_ptr[c], w->wpb);
    need = std::max(need, t);
  }
  if (d.wp_spmv.wpb > 0 && d.nc > 0) need = std::max<int64_t>(need, warp_grid(d.tile_ptr[d.nc], d.wp_spmv.wpb));
  return need;
}

void enqueue_fwd_warp(const DeviceLayout &d, int prec, const double *r, bool check_done, cudaStream_t s) {
  const WarpPlan &w = plan_of(d, true, prec);
  for (int c = 0; c < d.nc; ++c) {
    const unsigned grid = warp_grid(d.tile_ptr[c + 1] - d.tile_ptr[c], w.wpb);
    const size_t sm = (size_t)w.wpb * w.warp_bytes;
    if (prec == HBMC_PREC_F64)
      k_fwd_w<double, double><<<grid, 32 * w.wpb, sm, s>>>(warp_args<double>(d, true, c, w), r, d.y, d.sc, check_done ? 1 : 0);
    else
      k_fwd_w<float, float><<<grid, 32 * w.wpb, sm, s>>>(warp_args<float>(d, true, c, w), r, d.y32, d.sc, check_done ? 1 : 0);
  }
}

void enqueue_bwd_warp(const DeviceLayout &d, int prec, const double *r, int dot_mode, bool check_done, cudaStream_t s) {
  const WarpPlan &w = plan_of(d, false, prec);
  int64_t total = 0;
  for (int c = 0; c < d.nc; ++c) total += warp_grid(d.tile_ptr[c + 1] - d.tile_ptr[c], w.wpb);
  int64_t off = 0;
  const size_t sm = (size_t)w.wpb * w.warp_bytes;
  for (int c = d.nc - 1; c >= 0; --c) {
    const unsigned grid = warp_grid(d.tile_ptr[c + 1] - d.tile_ptr[c], w.wpb);
    const int last = c == 0;
    if (prec == HBMC_PREC_F64)
      k_bwd_w<double, double><<<grid, 32 * w.wpb, sm, s>>>(warp_args<double>(d, false, c, w), d.y, d.z, d.z32, r, d.sc,
                                                           check_done ? 1 : 0, dot_mode, d.part, off, last, total);
    else
      k_bwd_w<float, float><<<grid, 32 * w.wpb, sm, s>>>(warp_args<float>(d, false, c, w), d.y32, d.z, d.z32, r, d.sc,
                                                         check_done ? 1 : 0, dot_mode, d.part, off, last, total);
    off += grid;
  }
}

void enqueue_spmv_warp(const DeviceLayout &d, const double *p, double *q, bool dot, cudaStream_t s) {
  const WarpPlan &w = d.wp_spmv;
  const int64_t units = d.tile_ptr[d.nc];
  const unsigned grid = warp_grid(units, w.wpb);
  const size_t sm = (size_t)w.wpb * w.warp_bytes;
  if (dot)
    k_spmv_w<true><<<grid, 32 * w.wpb, sm, s>>>(d.rec_a, d.rec_ints, d.a_col, d.a_val, d.bs, units, w.off_t,
                                                w.warp_bytes, p, q, d.part, d.sc);
  else
    k_spmv_w<false><<<grid, 32 * w.wpb, sm, s>>>(d.rec_a, d.rec_ints, d.a_col, d.a_val, d.bs, units, w.off_t,
                                                 w.warp_bytes, p, q, d.part, d.sc);
}

}  // namespace hbmc

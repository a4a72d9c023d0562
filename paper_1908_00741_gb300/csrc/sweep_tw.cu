// Substitution sweeps, one warp per level-1 block with its contiguous
// operands moved by bulk copy (w = 32, bs = 4 or 8; other shapes use
// sweep_warp.cu).
//
// A warp's work for its level-1 block ("unit", Eq. "BAMC3") is laid out to
// need few dependent trips to memory:
//   trip 1  lane 0 starts 1-D bulk copies (cp.async.bulk, completing on a
//           per-warp mbarrier) of the unit's right-hand-side and dinv
//           segments -- their addresses follow from the unit index alone --
//           while every lane loads the unit's record into registers;
//   trip 2  with the record known, lane 0 adds bulk copies of the unit's
//           same-block coefficients and their step indices, and the lanes
//           gather the other-color couplings of Eq. "for3" (coefficient,
//           column and vector entry, kChunk per lane at a time);
// then each lane runs its bs-step chain (Eqs. "y2-2", "y2-3") out of shared
// memory and stores its rows.  Nothing is staged through registers.  The
// column indices stay out of shared memory on purpose: with them a warp
// needs about 11 KB (FP64, bs 8) and only 5 CUDA blocks of 4 warps fit on an
// SM, so the 27 units per SM of a 128^3 color run in two waves; without
// them 7 blocks fit and one wave covers them.  Per-row term order is the
// layout's (other colors first, then the same block, farthest column from
// the diagonal first), identical to the oracle's.
//
// With w = 32 every run starts and ends on a multiple of 32 entries and every
// unit covers 32 * bs consecutive rows, so each copy's addresses and size are
// multiples of 16 bytes as bulk copies require.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "device_util.cuh"
#include "hbmc_internal.h"
#include "kernels.h"
#include "warp_common.cuh"

namespace hbmc {
namespace {

constexpr int kTwWarps = 4;
constexpr int kTwMinBlocks = 7;  // resident CUDA blocks per SM the register budget is cut for
constexpr uint64_t kTwWaitNs = 4000000000ull;
constexpr size_t kTwSmemBudget = 200 * 1024;
constexpr uint32_t kRecOff = 16;  // record after the 8-byte mbarrier; at most 64 ints

template <typename T>
struct TwArgs {
  const int32_t *rec;
  const int32_t *o_col;
  const T *o_val;
  const uint8_t *i_m;
  const T *i_val;
  const T *dinv;
  int rec_ints;
  int64_t tile0, ntiles;
  uint32_t off_ts, off_tin, off_ds, off_iv, off_im, warp_bytes;
};

// record int k (k < 64) held by lane k % 32 in r0 (k < 32) or r1
__device__ __forceinline__ int32_t rec_at(int32_t r0, int32_t r1, int k) {
  const int32_t a = __shfl_sync(0xffffffffu, r0, k & 31);
  const int32_t b = __shfl_sync(0xffffffffu, r1, k & 31);
  return k < 32 ? a : b;
}

template <int BS, bool FWD, typename T, typename IN, typename G, typename OUT>
__device__ __forceinline__ void tw_unit(const TwArgs<T> &a, unsigned char *ws, int lane, int64_t u, const IN *in,
                                        const G *gsrc, OUT *out, const double *r, bool dot, double &rz, Scalars *sc,
                                        float *out32 = nullptr) {
  constexpr uint32_t R = (uint32_t)BS * 32;
  uint64_t *bar = reinterpret_cast<uint64_t *>(ws);
  int32_t *rs = reinterpret_cast<int32_t *>(ws + kRecOff);
  T *ts = reinterpret_cast<T *>(ws + a.off_ts);
  IN *tin = reinterpret_cast<IN *>(ws + a.off_tin);  // == ts when IN is T
  T *ds = reinterpret_cast<T *>(ws + a.off_ds);
  T *iv = reinterpret_cast<T *>(ws + a.off_iv);
  uint8_t *im = ws + a.off_im;
  const int64_t row0 = u * (int64_t)R;
  // trip 1
  if (lane == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
    mbar_expect_tx(bar, R * (uint32_t)(sizeof(IN) + sizeof(T)));
    tma_load_1d(tin, in + row0, R * (uint32_t)sizeof(IN), bar);
    tma_load_1d(ds, a.dinv + row0, R * (uint32_t)sizeof(T), bar);
  }
  const int32_t *rc = a.rec + u * a.rec_ints;
  const int32_t r0 = lane < a.rec_ints ? rc[lane] : 0;
  const int32_t r1 = lane + 32 < a.rec_ints ? rc[lane + 32] : 0;
  const int olen = rec_at(r0, r1, 0), ilen = rec_at(r0, r1, 1);
  const int64_t obeg = (int64_t)(((uint64_t)(uint32_t)rec_at(r0, r1, 3) << 32) | (uint32_t)rec_at(r0, r1, 2));
  const int64_t ibeg = (int64_t)(((uint64_t)(uint32_t)rec_at(r0, r1, 5) << 32) | (uint32_t)rec_at(r0, r1, 4));
  // trip 2 (FP32: the other-color run is also prefetched into L2, so that
  // its later chunks come from L2; measured 22.2 -> 20.7 us for the 128^3
  // forward sweep, no gain in FP64)
  if (lane == 0) {
    if constexpr (sizeof(T) == 4) {
      if (olen > 0) {
        prefetch_l2(a.o_col + obeg, (uint32_t)olen * 4u);
        prefetch_l2(a.o_val + obeg, (uint32_t)olen * (uint32_t)sizeof(T));
      }
    }
    mbar_arrive_expect_tx(bar, (uint32_t)ilen * (uint32_t)(sizeof(T) + 1));
    if (ilen > 0) {
      tma_load_1d(iv, a.i_val + ibeg, (uint32_t)ilen * (uint32_t)sizeof(T), bar);
      tma_load_1d(im, a.i_m + ibeg, (uint32_t)ilen, bar);
    }
  }
  if (lane < a.rec_ints) rs[lane] = r0;
  if (lane + 32 < a.rec_ints) rs[lane + 32] = r1;
  __syncwarp();
  const uint64_t deadline = global_ns() + kTwWaitNs;
  const bool ok = mbar_wait(bar, 0, deadline);
  if (!__all_sync(0xffffffffu, ok)) {
    if (lane == 0) {
      sc->timeout = 1;
      sc->done = 1;
    }
    mbar_wait(bar, 0, deadline + kTwWaitNs);  // let the copies land before the warp leaves
    return;
  }
  if constexpr (!std::is_same<IN, T>::value) {
#pragma unroll
    for (int l = 0; l < BS; ++l) ts[(l << 5) + lane] = cvt<T>(tin[(l << 5) + lane]);
  }
  // other-color couplings
  run_accumulate<T, G, true>(a.o_col, a.o_val, gsrc, obeg, olen, rs + 6, ts, lane);
  const int32_t *i_rel = rs + 7 + BS;
  double rv[BS];
  if (!FWD && dot) {
#pragma unroll
    for (int q = 0; q < BS; ++q) rv[q] = r[row0 + (q << 5) + lane];
  }
  // the bs-step chain: same-block couplings, then the dinv scaling
#pragma unroll
  for (int q = 0; q < BS; ++q) {
    const int lq = FWD ? q : BS - 1 - q;
    T acc = ts[(lq << 5) + lane];
    const int pe = i_rel[lq + 1];
    for (int p = i_rel[lq] + lane; p < pe; p += 32) acc = fma(-iv[p], ts[(im[p] << 5) + lane], acc);
    ts[(lq << 5) + lane] = acc * ds[(lq << 5) + lane];
  }
#pragma unroll
  for (int q = 0; q < BS; ++q) {
    const T yv = ts[(q << 5) + lane];
    out[row0 + (q << 5) + lane] = cvt<OUT>(yv);
    if constexpr (!FWD && sizeof(T) == 4) out32[row0 + (q << 5) + lane] = yv;
    if (!FWD && dot) rz = fma(rv[q], cvt<double>(yv), rz);
  }
}

template <typename T, typename Y, int BS>
__global__ void __launch_bounds__(32 * kTwWarps, kTwMinBlocks)
    k_fwd_tw(const TwArgs<T> a, const double *__restrict__ r, Y *y, Scalars *sc, int check_done) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (check_done && sc->done) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t u = a.tile0 + (int64_t)blockIdx.x * kTwWarps + warp;
  if (u >= a.tile0 + a.ntiles) return;
  double rz = 0.0;
  tw_unit<BS, true, T, double, Y, Y>(a, smem + (size_t)warp * a.warp_bytes, lane, u, r, y, y, nullptr, false, rz, sc);
}

template <typename T, typename Y, int BS>
__global__ void __launch_bounds__(32 * kTwWarps, kTwMinBlocks)
    k_bwd_tw(const TwArgs<T> a, const Y *__restrict__ yin, double *z, float *z32, const double *__restrict__ r,
             Scalars *sc, int check_done, int dot_mode, double *part, int64_t part_off, int last_launch,
             int64_t part_total) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (check_done && sc->done) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t u = a.tile0 + (int64_t)blockIdx.x * kTwWarps + warp;
  double rz = 0.0;
  if (u < a.tile0 + a.ntiles)
    tw_unit<BS, false, T, Y, T, double>(a, smem + (size_t)warp * a.warp_bytes, lane, u, yin, zgather<T>(z, z32), z,
                                        r, dot_mode != 0, rz, sc, z32);
  if (!dot_mode) return;
  rz_partial(rz, sc, dot_mode, part, part_off + blockIdx.x, last_launch, part_total, gridDim.x);
}

// The last color's forward sweep and the backward sweep's first color
// (the same color) in one pass: for the last color the backward sweep needs
// only the unit's own y (a last color has no later colors to gather from),
// so the warp that finishes the forward chain of a unit runs its backward
// chain at once, and y never goes to memory.  The backward same-block run
// reuses the forward one's shared memory: it is fetched by bulk copy once the
// forward chain is done (a third trip, instead of a second launch).  Every
// operation is the one the separate sweeps perform, in the same order.
template <int BS, typename T, typename Y>
__device__ __forceinline__ void fb_unit(const TwArgs<T> &af, const TwArgs<T> &ab, unsigned char *ws, int lane,
                                        int64_t u, const double *r, const Y *ysrc, double *z, float *z32, bool dot,
                                        double &rz, Scalars *sc) {
  constexpr uint32_t R = (uint32_t)BS * 32;
  uint64_t *bar = reinterpret_cast<uint64_t *>(ws);
  int32_t *rs = reinterpret_cast<int32_t *>(ws + kRecOff);
  T *ts = reinterpret_cast<T *>(ws + af.off_ts);
  double *tin = reinterpret_cast<double *>(ws + af.off_tin);  // == ts in FP64
  T *ds = reinterpret_cast<T *>(ws + af.off_ds);
  T *iv = reinterpret_cast<T *>(ws + af.off_iv);
  uint8_t *im = ws + af.off_im;
  const int64_t row0 = u * (int64_t)R;
  // trip 1: r and dinv (dinv is the same array in both directions for IC(0))
  if (lane == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
    mbar_expect_tx(bar, R * (uint32_t)(sizeof(double) + sizeof(T)));
    tma_load_1d(tin, r + row0, R * 8u, bar);
    tma_load_1d(ds, af.dinv + row0, R * (uint32_t)sizeof(T), bar);
  }
  const int32_t *rcf = af.rec + u * af.rec_ints, *rcb = ab.rec + u * ab.rec_ints;
  const int32_t f0 = lane < af.rec_ints ? rcf[lane] : 0, f1 = lane + 32 < af.rec_ints ? rcf[lane + 32] : 0;
  const int32_t b0 = lane < ab.rec_ints ? rcb[lane] : 0, b1 = lane + 32 < ab.rec_ints ? rcb[lane + 32] : 0;
  const int olen = rec_at(f0, f1, 0), ilen = rec_at(f0, f1, 1);
  const int64_t obeg = (int64_t)(((uint64_t)(uint32_t)rec_at(f0, f1, 3) << 32) | (uint32_t)rec_at(f0, f1, 2));
  const int64_t ibeg = (int64_t)(((uint64_t)(uint32_t)rec_at(f0, f1, 5) << 32) | (uint32_t)rec_at(f0, f1, 4));
  const int olen_b = rec_at(b0, b1, 0), ilen_b = rec_at(b0, b1, 1);
  const int64_t obeg_b = (int64_t)(((uint64_t)(uint32_t)rec_at(b0, b1, 3) << 32) | (uint32_t)rec_at(b0, b1, 2));
  const int64_t ibeg_b = (int64_t)(((uint64_t)(uint32_t)rec_at(b0, b1, 5) << 32) | (uint32_t)rec_at(b0, b1, 4));
  // trip 2: the forward same-block run (and, FP32, the other-color run into L2)
  if (lane == 0) {
    if constexpr (sizeof(T) == 4) {
      if (olen > 0) {
        prefetch_l2(af.o_col + obeg, (uint32_t)olen * 4u);
        prefetch_l2(af.o_val + obeg, (uint32_t)olen * (uint32_t)sizeof(T));
      }
    }
    mbar_arrive_expect_tx(bar, (uint32_t)ilen * (uint32_t)(sizeof(T) + 1));
    if (ilen > 0) {
      tma_load_1d(iv, af.i_val + ibeg, (uint32_t)ilen * (uint32_t)sizeof(T), bar);
      tma_load_1d(im, af.i_m + ibeg, (uint32_t)ilen, bar);
    }
  }
  if (lane < af.rec_ints) rs[lane] = f0;
  if (lane + 32 < af.rec_ints) rs[lane + 32] = f1;
  __syncwarp();
  const uint64_t deadline = global_ns() + kTwWaitNs;
  if (!__all_sync(0xffffffffu, mbar_wait(bar, 0, deadline))) {
    if (lane == 0) {
      sc->timeout = 1;
      sc->done = 1;
    }
    mbar_wait(bar, 0, deadline + kTwWaitNs);  // let the copies land before the warp leaves
    return;
  }
  if constexpr (!std::is_same<T, double>::value) {
#pragma unroll
    for (int l = 0; l < BS; ++l) ts[(l << 5) + lane] = cvt<T>(tin[(l << 5) + lane]);
  }
  run_accumulate<T, Y, true>(af.o_col, af.o_val, ysrc, obeg, olen, rs + 6, ts, lane);
  {
    const int32_t *i_rel = rs + 7 + BS;
#pragma unroll
    for (int q = 0; q < BS; ++q) {
      T acc = ts[(q << 5) + lane];
      const int pe = i_rel[q + 1];
      for (int p = i_rel[q] + lane; p < pe; p += 32) acc = fma(-iv[p], ts[(im[p] << 5) + lane], acc);
      ts[(q << 5) + lane] = acc * ds[(q << 5) + lane];
    }
  }
  // trip 3: the backward same-block run into the same buffers, the backward
  // record into rs
  __syncwarp();
  if (lane == 0) {
    fence_proxy_async();
    mbar_arrive_expect_tx(bar, (uint32_t)ilen_b * (uint32_t)(sizeof(T) + 1));
    if (ilen_b > 0) {
      tma_load_1d(iv, ab.i_val + ibeg_b, (uint32_t)ilen_b * (uint32_t)sizeof(T), bar);
      tma_load_1d(im, ab.i_m + ibeg_b, (uint32_t)ilen_b, bar);
    }
  }
  if (lane < ab.rec_ints) rs[lane] = b0;
  if (lane + 32 < ab.rec_ints) rs[lane + 32] = b1;
  double rv[BS];
  if (dot) {
#pragma unroll
    for (int q = 0; q < BS; ++q) rv[q] = r[row0 + (q << 5) + lane];
  }
  __syncwarp();
  // a last color has no later colors: its backward other-color run is empty
  run_accumulate<T, T, true>(ab.o_col, ab.o_val, zgather<T>(z, z32), obeg_b, olen_b, rs + 6, ts, lane);
  if (!__all_sync(0xffffffffu, mbar_wait(bar, 1, deadline + kTwWaitNs))) {
    if (lane == 0) {
      sc->timeout = 1;
      sc->done = 1;
    }
    mbar_wait(bar, 1, deadline + 2 * kTwWaitNs);
    return;
  }
  {
    const int32_t *i_rel = rs + 7 + BS;
#pragma unroll
    for (int q = 0; q < BS; ++q) {
      const int lq = BS - 1 - q;
      T acc = ts[(lq << 5) + lane];
      const int pe = i_rel[lq + 1];
      for (int p = i_rel[lq] + lane; p < pe; p += 32) acc = fma(-iv[p], ts[(im[p] << 5) + lane], acc);
      ts[(lq << 5) + lane] = acc * ds[(lq << 5) + lane];
    }
  }
#pragma unroll
  for (int q = 0; q < BS; ++q) {
    const T zv = ts[(q << 5) + lane];
    const double zd = cvt<double>(zv);
    z[row0 + (q << 5) + lane] = zd;
    if constexpr (sizeof(T) == 4) z32[row0 + (q << 5) + lane] = zv;
    if (dot) rz = fma(rv[q], zd, rz);
  }
}

template <typename T, typename Y, int BS>
__global__ void __launch_bounds__(32 * kTwWarps, kTwMinBlocks)
    k_fb_tw(const TwArgs<T> af, const TwArgs<T> ab, const double *__restrict__ r, const Y *ysrc, double *z,
            float *z32, Scalars *sc, int check_done, int dot_mode, double *part, int64_t part_off, int last_launch,
            int64_t part_total) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (check_done && sc->done) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t u = af.tile0 + (int64_t)blockIdx.x * kTwWarps + warp;
  double rz = 0.0;
  if (u < af.tile0 + af.ntiles)
    fb_unit<BS, T, Y>(af, ab, smem + (size_t)warp * af.warp_bytes, lane, u, r, ysrc, z, z32, dot_mode != 0, rz, sc);
  if (!dot_mode) return;
  rz_partial(rz, sc, dot_mode, part, part_off + blockIdx.x, last_launch, part_total, gridDim.x);
}

uint32_t a16(uint64_t v) { return (uint32_t)((v + 15) & ~uint64_t(15)); }

template <typename T>
TwArgs<T> tw_args(const DeviceLayout &d, bool fwd, int c, const TwPlan &p) {
  TwArgs<T> a;
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
  a.tile0 = d.tile_ptr[c];
  a.ntiles = d.tile_ptr[c + 1] - d.tile_ptr[c];
  a.off_ts = p.off_ts;
  a.off_tin = p.off_tin;
  a.off_ds = p.off_ds;
  a.off_iv = p.off_iv;
  a.off_im = p.off_im;
  a.warp_bytes = p.warp_bytes;
  return a;
}

// Forward sweeps read the double right-hand side r; in FP32 it lands in a
// region of its own and is narrowed into ts.  Every other case copies the
// input straight into ts.
TwPlan plan_one(int bs, bool fwd, int rec_ints, int64_t max_i, size_t tsize) {
  TwPlan p;
  const uint64_t R = (uint64_t)bs * 32;
  p.off_ts = a16(kRecOff + 4ull * 64);
  uint64_t next = p.off_ts + R * tsize;
  p.off_tin = p.off_ts;
  if (fwd && tsize != 8) {
    p.off_tin = a16(next);
    next = p.off_tin + R * 8;
  }
  p.off_ds = a16(next);
  p.off_iv = a16(p.off_ds + R * tsize);
  p.off_im = a16(p.off_iv + (uint64_t)max_i * tsize);
  p.warp_bytes = (uint32_t)((p.off_im + (uint64_t)max_i + 127) & ~uint64_t(127));
  p.ok = rec_ints <= 64 && (uint64_t)kTwWarps * p.warp_bytes <= kTwSmemBudget;
  return p;
}

const TwPlan &tw_plan(const DeviceLayout &d, bool fwd, int prec) {
  return prec == HBMC_PREC_F64 ? (fwd ? d.tw_f64_f : d.tw_f64_b) : (fwd ? d.tw_f32_f : d.tw_f32_b);
}

unsigned tw_grid(const DeviceLayout &d, int c) {
  return (unsigned)((d.tile_ptr[c + 1] - d.tile_ptr[c] + kTwWarps - 1) / kTwWarps);
}

template <typename T, typename Y, int BS>
void launch_fwd(const DeviceLayout &d, int c, const double *r, Y *y, bool check_done, cudaStream_t s,
                const TwPlan &p) {
  k_fwd_tw<T, Y, BS><<<tw_grid(d, c), 32 * kTwWarps, (size_t)kTwWarps * p.warp_bytes, s>>>(
      tw_args<T>(d, true, c, p), r, y, d.sc, check_done ? 1 : 0);
}

template <typename T, typename Y, int BS>
void launch_bwd(const DeviceLayout &d, int c, const Y *yin, const double *r, int dot_mode, bool check_done,
                int64_t part_off, bool last, int64_t part_total, cudaStream_t s, const TwPlan &p) {
  k_bwd_tw<T, Y, BS><<<tw_grid(d, c), 32 * kTwWarps, (size_t)kTwWarps * p.warp_bytes, s>>>(
      tw_args<T>(d, false, c, p), yin, d.z, d.z32, r, d.sc, check_done ? 1 : 0, dot_mode, d.part, part_off,
      last ? 1 : 0, part_total);
}

template <typename K>
cudaError_t allow(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTwSmemBudget);
}

}  // namespace

void plan_tw_kernels(const HostLayout &h, DeviceLayout &d) {
  d.tw_f64_f = plan_one(h.bs, true, h.rec_ints, h.max_i_f, 8);
  d.tw_f64_b = plan_one(h.bs, false, h.rec_ints, h.max_i_b, 8);
  d.tw_f32_f = plan_one(h.bs, true, h.rec_ints, h.max_i_f, 4);
  d.tw_f32_b = plan_one(h.bs, false, h.rec_ints, h.max_i_b, 4);
  // the same-block buffers hold either direction's run
  const int64_t mi = std::max(h.max_i_f, h.max_i_b);
  d.tw_fb_f64 = plan_one(h.bs, true, h.rec_ints, mi, 8);
  d.tw_fb_f32 = plan_one(h.bs, true, h.rec_ints, mi, 4);
}

// The fused last-color pass: both directions on the bulk-copy warp kernels
// for the last color, one dinv for both (IC(0)), and its plan fits.
bool fb_tw_usable(const DeviceLayout &d, int prec) {
  if (d.nc < 1 || !tw_usable(d, true, prec) || !tw_usable(d, false, prec)) return false;
  if (dag_selected(d, prec)) return false;
  if (d.dinvb != d.dinv || d.dinvb32 != d.dinv32) return false;
  const int c = d.nc - 1;
  if (wide_usable(d, true, prec) && wide_preferred(d, true, c)) return false;
  if (wide_usable(d, false, prec) && wide_preferred(d, false, c)) return false;
  return (prec == HBMC_PREC_F64 ? d.tw_fb_f64 : d.tw_fb_f32).ok;
}

template <typename T, typename Y, int BS>
static void launch_fb(const DeviceLayout &d, const double *r, const Y *ysrc, int dot_mode, bool check_done,
                      int64_t part_off, bool last, int64_t part_total, cudaStream_t s) {
  const int c = d.nc - 1;
  const TwPlan &pf = sizeof(T) == 8 ? d.tw_fb_f64 : d.tw_fb_f32;
  const TwPlan &pb = sizeof(T) == 8 ? d.tw_f64_b : d.tw_f32_b;
  k_fb_tw<T, Y, BS><<<tw_grid(d, c), 32 * kTwWarps, (size_t)kTwWarps * pf.warp_bytes, s>>>(
      tw_args<T>(d, true, c, pf), tw_args<T>(d, false, c, pb), r, ysrc, d.z, d.z32, d.sc, check_done ? 1 : 0,
      dot_mode, d.part, part_off, last ? 1 : 0, part_total);
}

void launch_fb_tw_last(const DeviceLayout &d, int prec, const double *r, int dot_mode, bool check_done,
                       int64_t part_off, bool last, int64_t part_total, cudaStream_t s) {
  if (tw_color_grid(d, d.nc - 1) == 0) return;
  if (prec == HBMC_PREC_F64) {
    if (d.bs == 8) launch_fb<double, double, 8>(d, r, d.y, dot_mode, check_done, part_off, last, part_total, s);
    else launch_fb<double, double, 4>(d, r, d.y, dot_mode, check_done, part_off, last, part_total, s);
  } else {
    if (d.bs == 8) launch_fb<float, float, 8>(d, r, d.y32, dot_mode, check_done, part_off, last, part_total, s);
    else launch_fb<float, float, 4>(d, r, d.y32, dot_mode, check_done, part_off, last, part_total, s);
  }
}

cudaError_t setup_tw_kernels() {
  cudaError_t e;
  if ((e = allow(k_fwd_tw<double, double, 4>)) || (e = allow(k_fwd_tw<double, double, 8>)) ||
      (e = allow(k_fwd_tw<float, float, 4>)) || (e = allow(k_fwd_tw<float, float, 8>)) ||
      (e = allow(k_bwd_tw<double, double, 4>)) || (e = allow(k_bwd_tw<double, double, 8>)) ||
      (e = allow(k_bwd_tw<float, float, 4>)) || (e = allow(k_bwd_tw<float, float, 8>)) ||
      (e = allow(k_fb_tw<double, double, 4>)) || (e = allow(k_fb_tw<double, double, 8>)) ||
      (e = allow(k_fb_tw<float, float, 4>)) || (e = allow(k_fb_tw<float, float, 8>)))
    return e;
  return cudaSuccess;
}

bool tw_usable(const DeviceLayout &d, bool fwd, int prec) {
  return (d.sweep_kernel == 0 || d.sweep_kernel == 5) && d.w == 32 && (d.bs == 4 || d.bs == 8) && d.rec_f &&
         tw_plan(d, fwd, prec).ok;
}

int64_t tw_partials_needed(const DeviceLayout &d) {
  int64_t t = 0;
  for (int c = 0; c < d.nc; ++c) t += tw_grid(d, c);
  return t;
}

unsigned tw_color_grid(const DeviceLayout &d, int c) { return tw_grid(d, c); }

void launch_fwd_tw_color(const DeviceLayout &d, int prec, int c, const double *r, bool check_done, cudaStream_t s) {
  const TwPlan &p = tw_plan(d, true, prec);
  if (prec == HBMC_PREC_F64) {
    if (d.bs == 4) launch_fwd<double, double, 4>(d, c, r, d.y, check_done, s, p);
    else launch_fwd<double, double, 8>(d, c, r, d.y, check_done, s, p);
  } else {
    if (d.bs == 4) launch_fwd<float, float, 4>(d, c, r, d.y32, check_done, s, p);
    else launch_fwd<float, float, 8>(d, c, r, d.y32, check_done, s, p);
  }
}

void launch_bwd_tw_color(const DeviceLayout &d, int prec, int c, const double *r, int dot_mode, bool check_done,
                         int64_t part_off, bool last, int64_t part_total, cudaStream_t s) {
  const TwPlan &p = tw_plan(d, false, prec);
  if (prec == HBMC_PREC_F64) {
    if (d.bs == 4) launch_bwd<double, double, 4>(d, c, d.y, r, dot_mode, check_done, part_off, last, part_total, s, p);
    else launch_bwd<double, double, 8>(d, c, d.y, r, dot_mode, check_done, part_off, last, part_total, s, p);
  } else {
    if (d.bs == 4) launch_bwd<float, float, 4>(d, c, d.y32, r, dot_mode, check_done, part_off, last, part_total, s, p);
    else launch_bwd<float, float, 8>(d, c, d.y32, r, dot_mode, check_done, part_off, last, part_total, s, p);
  }
}

}  // namespace hbmc

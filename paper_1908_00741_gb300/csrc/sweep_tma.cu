// Substitution sweeps as persistent, warp-specialized CUDA blocks fed by TMA.
//
// One launch per color (Section 4.3.3: the n_c - 1 synchronizations become
// kernel boundaries).  Every level-1 block of the color (Eq. "BAMC3") is a
// unit of work; a CUDA block takes units blockIdx.x, blockIdx.x + gridDim.x,
// ...  Warp 0 is the producer: one lane issues 1-D TMA bulk copies
// (cp.async.bulk + mbarrier) of everything of a unit that lies contiguously
// in memory -- its slice offsets, the right-hand side and dinv segments and
// the coefficient runs -- into a ring of shared-memory stages, running up to
// `stages` units ahead.  Warps 1..8 consume: the couplings to other colors
// (Eq. "for3"), one thread per row, gather the only irregular operands; one
// warp then runs the bs-step chain of Eqs. "y2-2"/"y2-3" for the w = 32 BMC
// blocks of the unit in shared memory; finally all consumers store the unit.
//
// Every wait on an mbarrier is bounded by the global timer; on expiry the
// kernel records a timeout in the solve's scalars, stops computing, lets
// its bulk copies in flight land, and exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "device_util.cuh"
#include "hbmc_internal.h"
#include "kernels.h"

namespace hbmc {
namespace {

constexpr int kConsWarps = 8;
constexpr int kTmaThreads = 32 * (kConsWarps + 1);
constexpr int kConsThreads = 32 * kConsWarps;
constexpr int kMaxStages = 4;
constexpr uint64_t kWaitNs = 4000000000ull;  // 4 s
constexpr size_t kTmaSmemBudget = 200 * 1024;

template <typename T>
struct TmaSweep {
  const int32_t *rec;  // per-unit records, rec_ints int32 each
  const int32_t *o_col;
  const T *o_val;
  const uint8_t *i_m;
  const T *i_val;
  const T *dinv;
  int bs, rec_ints, stages;
  int64_t tile0, ntiles;
  uint32_t off_in, off_dinv, off_aux, off_ocol, off_oval, off_ival, off_im, stage_bytes;
};

// Record layout (int32): [0] o_len, [1] i_len, [2..3] o_begin, [4..5] i_begin,
// [6 .. 6+bs] o_rel, [7+bs .. 7+2bs] i_rel (slice offsets inside the runs).
__device__ __forceinline__ int64_t rec_i64(const int32_t *r, int k) {
  return (int64_t)(((uint64_t)(uint32_t)r[k + 1] << 32) | (uint64_t)(uint32_t)r[k]);
}

__device__ __forceinline__ void note_timeout(Scalars *sc, volatile int *abort_flag) {
  *abort_flag = 1;
  if (sc) {
    sc->timeout = 1;
    sc->done = 1;
  }
}

// Producer loop (one lane).  `in` is the per-row input segment base, `aux`
// an optional second per-row double segment (the backward sweep's r).
template <typename T, typename IN>
__device__ __forceinline__ void produce(const TmaSweep<T> &a, unsigned char *smem, uint64_t *full, uint64_t *empty,
                        const IN *in, const double *aux, Scalars *sc, volatile int *abort_flag,
                        uint64_t deadline) {
  const int R = a.bs * 32;
  const uint32_t rec_bytes = (uint32_t)a.rec_ints * 4u;
  int k = 0;
  for (int64_t u = a.tile0 + blockIdx.x; u < a.tile0 + a.ntiles; u += gridDim.x, ++k) {
    const int st = k % a.stages;
    const uint32_t ph = (uint32_t)(k / a.stages) & 1u;
    if (*abort_flag) break;
    if (k >= a.stages && !mbar_wait(&empty[st], ph ^ 1u, deadline)) {
      note_timeout(sc, abort_flag);
      break;
    }
    const int32_t *rc = a.rec + u * a.rec_ints;
    const int32_t olen = rc[0], ilen = rc[1];
    const int64_t obeg = rec_i64(rc, 2), ibeg = rec_i64(rc, 4);
    unsigned char *sb = smem + (size_t)st * a.stage_bytes;
    uint32_t bytes = rec_bytes + (uint32_t)(R * sizeof(IN)) + (uint32_t)(R * sizeof(T)) +
                     (uint32_t)olen * (uint32_t)(4 + sizeof(T)) + (uint32_t)ilen * (uint32_t)(1 + sizeof(T));
    if (aux) bytes += (uint32_t)(R * sizeof(double));
    mbar_arrive_expect_tx(&full[st], bytes);
    tma_load_1d(sb, rc, rec_bytes, &full[st]);
    tma_load_1d(sb + a.off_in, in + u * R, (uint32_t)(R * sizeof(IN)), &full[st]);
    tma_load_1d(sb + a.off_dinv, a.dinv + u * R, (uint32_t)(R * sizeof(T)), &full[st]);
    if (aux) tma_load_1d(sb + a.off_aux, aux + u * R, (uint32_t)(R * sizeof(double)), &full[st]);
    if (olen > 0) {
      tma_load_1d(sb + a.off_ocol, a.o_col + obeg, (uint32_t)olen * 4u, &full[st]);
      tma_load_1d(sb + a.off_oval, a.o_val + obeg, (uint32_t)olen * (uint32_t)sizeof(T), &full[st]);
    }
    if (ilen > 0) {
      tma_load_1d(sb + a.off_ival, a.i_val + ibeg, (uint32_t)ilen * (uint32_t)sizeof(T), &full[st]);
      tma_load_1d(sb + a.off_im, a.i_m + ibeg, (uint32_t)ilen, &full[st]);
    }
  }
  // let every copy still in flight land before the CTA may exit
  const int issued = k;
  for (int i = issued > a.stages ? issued - a.stages : 0; i < issued; ++i)
    if (!mbar_wait(&full[i % a.stages], (uint32_t)(i / a.stages) & 1u, deadline + kWaitNs)) break;
}

__device__ __forceinline__ void init_barriers(uint64_t *full, uint64_t *empty, int stages,
                                              volatile int *abort_flag) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsWarps);
    }
    *abort_flag = 0;
    mbar_fence_init();
  }
  __syncthreads();
}

template <typename T, typename Y>
__global__ void __launch_bounds__(kTmaThreads, 3)
    k_fwd_tma(const TmaSweep<T> a, const double *__restrict__ r, Y *y, Scalars *sc, int check_done) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t full[kMaxStages], empty[kMaxStages];
  __shared__ volatile int abort_flag;
  if (check_done && sc->done) return;
  init_barriers(full, empty, a.stages, &abort_flag);
  const uint64_t deadline = global_ns() + kWaitNs;
  const int R = a.bs * 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    if (lane == 0) produce<T, double>(a, smem, full, empty, r, nullptr, sc, &abort_flag, deadline);
    return;
  }
  T *tvbuf = reinterpret_cast<T *>(smem + (size_t)a.stages * a.stage_bytes);
  const int ct = threadIdx.x - 32;
  int k = 0;
  for (int64_t u = a.tile0 + blockIdx.x; u < a.tile0 + a.ntiles; u += gridDim.x, ++k) {
    const int st = k % a.stages;
    const uint32_t ph = (uint32_t)(k / a.stages) & 1u;
    if (!abort_flag && !mbar_wait(&full[st], ph, deadline)) note_timeout(sc, &abort_flag);
    const bool live = !abort_flag;
    const unsigned char *sb = smem + (size_t)st * a.stage_bytes;
    const int32_t *rec = reinterpret_cast<const int32_t *>(sb);
    const int32_t *o_rel = rec + 6, *i_rel = rec + 7 + a.bs;
    const double *rin = reinterpret_cast<const double *>(sb + a.off_in);
    const T *dv = reinterpret_cast<const T *>(sb + a.off_dinv);
    const int32_t *ocol = reinterpret_cast<const int32_t *>(sb + a.off_ocol);
    const T *oval = reinterpret_cast<const T *>(sb + a.off_oval);
    const T *ival = reinterpret_cast<const T *>(sb + a.off_ival);
    const uint8_t *im = sb + a.off_im;
    T *tv = tvbuf + (k & 1) * R;
    if (live) {
#pragma unroll 4
      for (int lr = ct; lr < R; lr += kConsThreads) {
        const int l = lr >> 5, j = lr & 31;
        T acc = (T)rin[lr];
        const int pe = o_rel[l + 1];
        for (int p = o_rel[l] + j; p < pe; p += 32) acc = fma(-oval[p], (T)y[ocol[p]], acc);
        tv[lr] = acc;
      }
    }
    named_sync(1, kConsThreads);
    if (live && warp == 1) {
      for (int l = 0; l < a.bs; ++l) {
        T acc = tv[(l << 5) + lane];
        const int pe = i_rel[l + 1];
        for (int p = i_rel[l] + lane; p < pe; p += 32) acc = fma(-ival[p], tv[(im[p] << 5) + lane], acc);
        tv[(l << 5) + lane] = acc * dv[(l << 5) + lane];
      }
    }
    named_sync(1, kConsThreads);
    if (lane == 0) mbar_arrive(&empty[st]);
    if (live) {
      Y *yo = y + u * R;
#pragma unroll 4
      for (int lr = ct; lr < R; lr += kConsThreads) yo[lr] = (Y)tv[lr];
    }
  }
}

// dot_mode as in the plain backward kernel: 0 none, 1 initial rho, 2 rho and
// beta; the launch of color 1 (last_launch) finishes the sum.
template <typename T, typename Y>
__global__ void __launch_bounds__(kTmaThreads, 3)
    k_bwd_tma(const TmaSweep<T> a, const Y *__restrict__ yin, double *z, float *z32, const double *__restrict__ r,
              Scalars *sc, int check_done, int dot_mode, double *part, int64_t part_off,
              int last_launch, int64_t part_total) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t full[kMaxStages], empty[kMaxStages];
  __shared__ volatile int abort_flag;
  if (check_done && sc->done) return;
  init_barriers(full, empty, a.stages, &abort_flag);
  const uint64_t deadline = global_ns() + kWaitNs;
  const int R = a.bs * 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double rz = 0.0;
  if (warp == 0) {
    if (lane == 0) produce<T, Y>(a, smem, full, empty, yin, dot_mode ? r : nullptr, sc, &abort_flag, deadline);
  } else {
    T *tvbuf = reinterpret_cast<T *>(smem + (size_t)a.stages * a.stage_bytes);
    const int ct = threadIdx.x - 32;
    int k = 0;
    for (int64_t u = a.tile0 + blockIdx.x; u < a.tile0 + a.ntiles; u += gridDim.x, ++k) {
      const int st = k % a.stages;
      const uint32_t ph = (uint32_t)(k / a.stages) & 1u;
      if (!abort_flag && !mbar_wait(&full[st], ph, deadline)) note_timeout(sc, &abort_flag);
      const bool live = !abort_flag;
      const unsigned char *sb = smem + (size_t)st * a.stage_bytes;
      const int32_t *rec = reinterpret_cast<const int32_t *>(sb);
      const int32_t *o_rel = rec + 6, *i_rel = rec + 7 + a.bs;
      const Y *yseg = reinterpret_cast<const Y *>(sb + a.off_in);
      const T *dv = reinterpret_cast<const T *>(sb + a.off_dinv);
      const double *rseg = reinterpret_cast<const double *>(sb + a.off_aux);
      const int32_t *ocol = reinterpret_cast<const int32_t *>(sb + a.off_ocol);
      const T *oval = reinterpret_cast<const T *>(sb + a.off_oval);
      const T *ival = reinterpret_cast<const T *>(sb + a.off_ival);
      const uint8_t *im = sb + a.off_im;
      T *tv = tvbuf + (k & 1) * R;
      if (live) {
#pragma unroll 4
        for (int lr = ct; lr < R; lr += kConsThreads) {
          const int l = lr >> 5, j = lr & 31;
          T acc = (T)yseg[lr];
          const int pe = o_rel[l + 1];
          const T *zg = zgather<T>(z, z32);
          for (int p = o_rel[l] + j; p < pe; p += 32) acc = fma(-oval[p], zg[ocol[p]], acc);
          tv[lr] = acc;
        }
      }
      named_sync(1, kConsThreads);
      if (live && warp == 1) {
        for (int l = a.bs - 1; l >= 0; --l) {
          T acc = tv[(l << 5) + lane];
          const int pe = i_rel[l + 1];
          for (int p = i_rel[l] + lane; p < pe; p += 32) acc = fma(-ival[p], tv[(im[p] << 5) + lane], acc);
          tv[(l << 5) + lane] = acc * dv[(l << 5) + lane];
        }
      }
      named_sync(1, kConsThreads);
      if (live) {
        double *zo = z + u * R;
#pragma unroll 4
        for (int lr = ct; lr < R; lr += kConsThreads) {
          const double zv = (double)tv[lr];
          zo[lr] = zv;
          if constexpr (sizeof(T) == 4) z32[u * R + lr] = tv[lr];
          if (dot_mode) rz = fma(rseg[lr], zv, rz);
        }
      }
      // the stage (r segment included) is read until here
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    }
  }
  if (!dot_mode) return;
  const double v = block_sum<kTmaThreads>(rz);
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
  const double rho_new = gather_partials<kTmaThreads>(part, part_total, 1, 0);
  if (threadIdx.x != 0) return;
  sc->cnt[CNT_RZ] = 0;
  sc->rho_new = rho_new;
  if (sc->timeout) return;
  if (!(rho_new > 0.0) || !finite(rho_new)) {
    sc->status = ST_BREAKDOWN;
    sc->done = 1;
    return;
  }
  if (dot_mode == 2) sc->beta = rho_new / sc->rho;
  sc->rho = rho_new;
}

template <typename T>
TmaSweep<T> tma_args(const DeviceLayout &d, bool fwd, int c) {
  const TmaPlan &pl = fwd ? d.tma_f : d.tma_b;
  const TmaLayout &L = sizeof(T) == 8 ? pl.f64 : pl.f32;
  TmaSweep<T> a;
  a.rec = pl.rec;
  a.rec_ints = pl.rec_ints;
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
  a.stages = L.stages;
  a.tile0 = d.tile_ptr[c];
  a.ntiles = d.tile_ptr[c + 1] - d.tile_ptr[c];
  a.off_in = L.off_in;
  a.off_dinv = L.off_dinv;
  a.off_aux = L.off_aux;
  a.off_ocol = L.off_ocol;
  a.off_oval = L.off_oval;
  a.off_ival = L.off_ival;
  a.off_im = L.off_im;
  a.stage_bytes = L.stage_bytes;
  return a;
}

size_t tma_smem(const DeviceLayout &d, const TmaLayout &L, size_t tsize) {
  return (size_t)L.stages * L.stage_bytes + 2 * (size_t)d.bs * 32 * tsize;
}

unsigned tma_grid(const DeviceLayout &d, const TmaLayout &L, int c) {
  const int64_t nt = d.tile_ptr[c + 1] - d.tile_ptr[c];
  const int64_t cap = (int64_t)d.sm_count * (L.ctas_per_sm > 0 ? L.ctas_per_sm : 1);
  return (unsigned)std::min<int64_t>(nt, cap);
}

uint32_t a16(uint64_t v) { return (uint32_t)((v + 15) & ~uint64_t(15)); }

// Stage layout for one direction and one value type.
TmaLayout plan_layout(int bs, int rec_ints, int64_t max_o, int64_t max_i, size_t tsize, size_t in_size,
                      bool aux) {
  TmaLayout L;
  const uint64_t R = (uint64_t)bs * 32;
  uint64_t off = a16((uint64_t)rec_ints * 4);
  L.off_in = (uint32_t)off;
  off = a16(off + R * in_size);
  L.off_dinv = (uint32_t)off;
  off = a16(off + R * tsize);
  L.off_aux = (uint32_t)off;
  if (aux) off = a16(off + R * 8);
  L.off_ocol = (uint32_t)off;
  off = a16(off + (uint64_t)max_o * 4);
  L.off_oval = (uint32_t)off;
  off = a16(off + (uint64_t)max_o * tsize);
  L.off_ival = (uint32_t)off;
  off = a16(off + (uint64_t)max_i * tsize);
  L.off_im = (uint32_t)off;
  off = off + (uint64_t)max_i;
  L.stage_bytes = (uint32_t)((off + 127) & ~uint64_t(127));
  const uint64_t work = 2 * R * tsize;
  L.stages = 0;
  for (int s = 3; s >= 2; --s)
    if ((uint64_t)s * L.stage_bytes + work <= kTmaSmemBudget) {
      L.stages = s;
      break;
    }
  return L;
}

template <typename K>
int occupancy(K kernel, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kTmaThreads, smem) != cudaSuccess) return 0;
  return n;
}

}  // namespace

// Host: per-unit records and stage layouts for both directions.  The TMA
// path needs w = 32 (every run then starts and ends on a 16-byte boundary)
// and runs that fit the shared-memory budget; otherwise the plain kernels run.
void plan_tma(const HostLayout &h, TmaPlan &pf, TmaPlan &pb, std::vector<int32_t> &rec_f,
              std::vector<int32_t> &rec_b) {
  pf = TmaPlan();
  pb = TmaPlan();
  rec_f.clear();
  rec_b.clear();
  if (h.w != 32 || h.ntiles == 0) return;
  const int bs = h.bs;
  const int rec_ints = (8 + 2 * bs + 3) / 4 * 4;
  for (int dir = 0; dir < 2; ++dir) {
    const std::vector<int64_t> &op = dir == 0 ? h.fo_ptr : h.bo_ptr;
    const std::vector<int64_t> &ip = dir == 0 ? h.fi_ptr : h.bi_ptr;
    std::vector<int32_t> &rec = dir == 0 ? rec_f : rec_b;
    TmaPlan &pl = dir == 0 ? pf : pb;
    rec.assign((size_t)h.ntiles * rec_ints, 0);
    int64_t max_o = 0, max_i = 0;
    for (int64_t u = 0; u < h.ntiles; ++u) {
      int32_t *rc = rec.data() + (size_t)u * rec_ints;
      const int64_t s0 = u * bs;
      const int64_t olen = op[s0 + bs] - op[s0], ilen = ip[s0 + bs] - ip[s0];
      max_o = std::max(max_o, olen);
      max_i = std::max(max_i, ilen);
      rc[0] = (int32_t)olen;
      rc[1] = (int32_t)ilen;
      rc[2] = (int32_t)(uint32_t)((uint64_t)op[s0] & 0xffffffffu);
      rc[3] = (int32_t)(uint32_t)((uint64_t)op[s0] >> 32);
      rc[4] = (int32_t)(uint32_t)((uint64_t)ip[s0] & 0xffffffffu);
      rc[5] = (int32_t)(uint32_t)((uint64_t)ip[s0] >> 32);
      for (int l = 0; l <= bs; ++l) {
        rc[6 + l] = (int32_t)(op[s0 + l] - op[s0]);
        rc[7 + bs + l] = (int32_t)(ip[s0 + l] - ip[s0]);
      }
    }
    pl.rec_ints = rec_ints;
    pl.max_o = max_o;
    pl.max_i = max_i;
    pl.f64 = plan_layout(bs, rec_ints, max_o, max_i, 8, dir == 0 ? 8 : 8, dir == 1);
    pl.f32 = plan_layout(bs, rec_ints, max_o, max_i, 4, dir == 0 ? 8 : 4, dir == 1);
  }
}

cudaError_t setup_tma_kernels(DeviceLayout &d) {
  cudaError_t e;
  const int cap = (int)kTmaSmemBudget + 16 * 1024;
  if ((e = cudaFuncSetAttribute(k_fwd_tma<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap))) return e;
  if ((e = cudaFuncSetAttribute(k_fwd_tma<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap))) return e;
  if ((e = cudaFuncSetAttribute(k_bwd_tma<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap))) return e;
  if ((e = cudaFuncSetAttribute(k_bwd_tma<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap))) return e;
  if (d.tma_f.rec) {
    if (d.tma_f.f64.stages) d.tma_f.f64.ctas_per_sm = occupancy(k_fwd_tma<double, double>, tma_smem(d, d.tma_f.f64, 8));
    if (d.tma_f.f32.stages) d.tma_f.f32.ctas_per_sm = occupancy(k_fwd_tma<float, float>, tma_smem(d, d.tma_f.f32, 4));
  }
  if (d.tma_b.rec) {
    if (d.tma_b.f64.stages) d.tma_b.f64.ctas_per_sm = occupancy(k_bwd_tma<double, double>, tma_smem(d, d.tma_b.f64, 8));
    if (d.tma_b.f32.stages) d.tma_b.f32.ctas_per_sm = occupancy(k_bwd_tma<float, float>, tma_smem(d, d.tma_b.f32, 4));
  }
  return cudaGetLastError();
}

bool tma_usable(const DeviceLayout &d, bool fwd, int prec) {
  if (!d.use_tma) return false;
  const TmaPlan &pl = fwd ? d.tma_f : d.tma_b;
  const TmaLayout &L = prec == HBMC_PREC_F64 ? pl.f64 : pl.f32;
  return pl.rec && L.stages >= 2 && L.ctas_per_sm > 0;
}

void enqueue_fwd_tma(const DeviceLayout &d, int prec, const double *r, bool check_done, cudaStream_t s) {
  for (int c = 0; c < d.nc; ++c) {
    if (prec == HBMC_PREC_F64) {
      const TmaSweep<double> a = tma_args<double>(d, true, c);
      k_fwd_tma<double, double><<<tma_grid(d, d.tma_f.f64, c), kTmaThreads, tma_smem(d, d.tma_f.f64, 8), s>>>(
          a, r, d.y, d.sc, check_done ? 1 : 0);
    } else {
      const TmaSweep<float> a = tma_args<float>(d, true, c);
      k_fwd_tma<float, float><<<tma_grid(d, d.tma_f.f32, c), kTmaThreads, tma_smem(d, d.tma_f.f32, 4), s>>>(
          a, r, d.y32, d.sc, check_done ? 1 : 0);
    }
  }
}

void enqueue_bwd_tma(const DeviceLayout &d, int prec, const double *r, int dot_mode, bool check_done,
                     cudaStream_t s) {
  const TmaLayout &L = prec == HBMC_PREC_F64 ? d.tma_b.f64 : d.tma_b.f32;
  int64_t total = 0;
  for (int c = 0; c < d.nc; ++c) total += tma_grid(d, L, c);
  int64_t off = 0;
  for (int c = d.nc - 1; c >= 0; --c) {
    const unsigned grid = tma_grid(d, L, c);
    const int last = c == 0;
    if (prec == HBMC_PREC_F64) {
      const TmaSweep<double> a = tma_args<double>(d, false, c);
      k_bwd_tma<double, double><<<grid, kTmaThreads, tma_smem(d, L, 8), s>>>(
          a, d.y, d.z, d.z32, r, d.sc, check_done ? 1 : 0, dot_mode, d.part, off, last, total);
    } else {
      const TmaSweep<float> a = tma_args<float>(d, false, c);
      k_bwd_tma<float, float><<<grid, kTmaThreads, tma_smem(d, L, 4), s>>>(
          a, d.y32, d.z, d.z32, r, d.sc, check_done ? 1 : 0, dot_mode, d.part, off, last, total);
    }
    off += grid;
  }
}

int64_t tma_partials_needed(const DeviceLayout &d) {
  int64_t need = 0;
  for (const TmaLayout *L : {&d.tma_b.f64, &d.tma_b.f32}) {
    int64_t t = 0;
    for (int c = 0; c < d.nc; ++c) t += tma_grid(d, *L, c);
    need = std::max(need, t);
  }
  return need;
}

}  // namespace hbmc

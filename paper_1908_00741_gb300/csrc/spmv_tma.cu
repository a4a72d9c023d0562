// SpMV q = A p (Section 4.3.2's SELL layout, slices of w = 32 rows) as a
// persistent, warp-specialized kernel fed by bulk copies, with the fused p.q
// and alpha = rho / p.q of the CG step.
//
// Work is cut into chunks of kSlices consecutive slices; their column
// indices and values are contiguous in the SELL arrays, and so is the chunk's
// segment of p.  Warp 0 is the producer: one lane issues three 1-D bulk
// copies (cp.async.bulk + mbarrier) per chunk into a ring of shared-memory
// stages, running up to `stages` chunks ahead.  Warps 1..kSlices consume: warp
// k takes slice k of the chunk, one thread per row, reads columns and values
// from shared memory and gathers p from global memory, kGather loads in
// flight per thread, then adds the terms in ascending column order from zero
// with fused multiply-adds -- the same order and operations as the oracle's
// SpMV.  Only the gathers wait on DRAM; everything regular streams through
// the copy engine without occupying registers.
//
// Every mbarrier wait is bounded by the global timer; on expiry the kernel
// records a timeout in the solve's scalars, stops computing, lets its copies
// in flight land, and exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "device_util.cuh"
#include "hbmc_internal.h"
#include "kernels.h"
#include "warp_common.cuh"

namespace hbmc {
namespace {

constexpr int kSlices = 8;                       // consumer warps = slices per chunk
constexpr int kSpThreads = 32 * (kSlices + 1);
constexpr int kGather = 8;
constexpr int kSpMaxStages = 4;
constexpr uint64_t kSpWaitNs = 4000000000ull;
constexpr size_t kSpSmemPerSm = 200 * 1024;     // stage rings of all CUDA blocks on one SM
constexpr int kSpMaxBlocksPerSm = 4;             // 4 x 288 threads x 40 registers fit an SM

struct SpArgs {
  const int64_t *a_ptr;
  const int32_t *a_col;
  const double *a_val;
  int64_t nslices, nchunks;
  int stages;
  uint32_t off_val, off_p, stage_bytes;
};

__device__ __forceinline__ void sp_timeout(Scalars *sc, volatile int *abort_flag) {
  *abort_flag = 1;
  sc->timeout = 1;
  sc->done = 1;
}

// One lane: copies of chunk after chunk into the stage ring.
__device__ __forceinline__ void sp_produce(const SpArgs &a, unsigned char *smem, uint64_t *full, uint64_t *empty,
                                           const double *p, Scalars *sc, volatile int *abort_flag,
                                           uint64_t deadline) {
  int k = 0;
  for (int64_t c = blockIdx.x; c < a.nchunks; c += gridDim.x, ++k) {
    const int st = k % a.stages;
    const uint32_t ph = (uint32_t)(k / a.stages) & 1u;
    if (*abort_flag) break;
    if (k >= a.stages && !mbar_wait(&empty[st], ph ^ 1u, deadline)) {
      sp_timeout(sc, abort_flag);
      break;
    }
    const int64_t s0 = c * kSlices, s1 = min(s0 + kSlices, a.nslices);
    const int64_t e0 = a.a_ptr[s0], e1 = a.a_ptr[s1];
    const uint32_t ne = (uint32_t)(e1 - e0), nr = (uint32_t)(s1 - s0) * 32u;
    unsigned char *sb = smem + (size_t)st * a.stage_bytes;
    mbar_arrive_expect_tx(&full[st], ne * 12u + nr * 8u);
    if (ne > 0) {
      tma_load_1d(sb, a.a_col + e0, ne * 4u, &full[st]);
      tma_load_1d(sb + a.off_val, a.a_val + e0, ne * 8u, &full[st]);
    }
    tma_load_1d(sb + a.off_p, p + s0 * 32, nr * 8u, &full[st]);
  }
  const int issued = k;
  for (int i = issued > a.stages ? issued - a.stages : 0; i < issued; ++i)
    if (!mbar_wait(&full[i % a.stages], (uint32_t)(i / a.stages) & 1u, deadline + kSpWaitNs)) break;
}

template <bool kDot>
__global__ void __launch_bounds__(kSpThreads, kSpMaxBlocksPerSm)
    k_spmv_tma(const SpArgs a, const double *p, double *q, double *part, Scalars *sc) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t full[kSpMaxStages], empty[kSpMaxStages];
  __shared__ volatile int abort_flag;
  if (kDot && sc->done) return;
  if (threadIdx.x == 0) {
    for (int s = 0; s < a.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kSlices);
    }
    abort_flag = 0;
    mbar_fence_init();
  }
  __syncthreads();
  const uint64_t deadline = global_ns() + kSpWaitNs;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double pq = 0.0;
  if (warp == 0) {
    if (lane == 0) sp_produce(a, smem, full, empty, p, sc, &abort_flag, deadline);
  } else {
    const int ws = warp - 1;
    int k = 0;
    for (int64_t c = blockIdx.x; c < a.nchunks; c += gridDim.x, ++k) {
      const int st = k % a.stages;
      const uint32_t ph = (uint32_t)(k / a.stages) & 1u;
      const int64_t s0 = c * kSlices, s = s0 + ws;
      const bool has = s < a.nslices;
      const int64_t base = a.a_ptr[s0];
      const int64_t sb_ = has ? a.a_ptr[s] : 0, se = has ? a.a_ptr[s + 1] : 0;
      if (!abort_flag && !mbar_wait(&full[st], ph, deadline)) sp_timeout(sc, &abort_flag);
      if (!abort_flag && has) {
        const unsigned char *sb = smem + (size_t)st * a.stage_bytes;
        const int32_t *col = reinterpret_cast<const int32_t *>(sb) + (sb_ - base) + lane;
        const double *val = reinterpret_cast<const double *>(sb + a.off_val) + (sb_ - base) + lane;
        const int width = (int)((se - sb_) >> 5);
        double acc = 0.0;
        for (int t0 = 0; t0 < width; t0 += kGather) {
          double g[kGather];
#pragma unroll
          for (int t = 0; t < kGather; ++t)
            if (t0 + t < width) g[t] = p[col[(t0 + t) << 5]];
#pragma unroll
          for (int t = 0; t < kGather; ++t)
            if (t0 + t < width) acc = fma(val[(t0 + t) << 5], g[t], acc);
        }
        const int64_t row = s * 32 + lane;
        q[row] = acc;
        if (kDot) pq = fma(reinterpret_cast<const double *>(sb + a.off_p)[ws * 32 + lane], acc, pq);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
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
  if (sc->timeout) return;
  if (!(s > 0.0) || !finite(s)) {
    sc->status = ST_BREAKDOWN;
    sc->done = 1;
    return;
  }
  sc->alpha = sc->rho / s;
}

uint32_t al16(uint64_t v) { return (uint32_t)((v + 15) & ~uint64_t(15)); }

}  // namespace

void plan_spmv_tma(const HostLayout &h, DeviceLayout &d) {
  SpmvPlan &P = d.sp;
  P = SpmvPlan();
  if (h.w != 32 || h.n_pad == 0) return;
  const int64_t nslices = h.n_pad / 32;
  int64_t max_e = 0;
  for (int64_t s0 = 0; s0 < nslices; s0 += kSlices)
    max_e = std::max(max_e, h.a_ptr[std::min(s0 + kSlices, nslices)] - h.a_ptr[s0]);
  P.off_val = al16((uint64_t)max_e * 4);
  P.off_p = al16(P.off_val + (uint64_t)max_e * 8);
  P.stage_bytes = (uint32_t)((P.off_p + (uint64_t)kSlices * 32 * 8 + 127) & ~uint64_t(127));
  P.nslices = nslices;
  P.nchunks = (nslices + kSlices - 1) / kSlices;
  // as many CUDA blocks per SM as keep at least two stages each: more
  // consumer warps keep more gathers in flight (measured at 128^3: 4 blocks
  // of 2 stages beat 2 blocks of 4 stages)
  for (int bpsm = kSpMaxBlocksPerSm; bpsm >= 2; --bpsm) {
    const int64_t st = (int64_t)(kSpSmemPerSm / bpsm) / P.stage_bytes;
    if (st >= 2) {
      P.stages = (int)std::min<int64_t>(st, kSpMaxStages);
      P.blocks_per_sm = bpsm;
      return;
    }
  }
}

cudaError_t setup_spmv_tma() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_spmv_tma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSpSmemPerSm)))
    return e;
  return cudaFuncSetAttribute(k_spmv_tma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSpSmemPerSm);
}

bool spmv_tma_usable(const DeviceLayout &d) { return d.sweep_kernel != 3 && d.w == 32 && d.sp.stages >= 2; }

static unsigned spmv_tma_grid(const DeviceLayout &d) {
  return (unsigned)std::min<int64_t>(d.sp.nchunks, (int64_t)d.sm_count * d.sp.blocks_per_sm);
}

int64_t spmv_tma_partials_needed(const DeviceLayout &d) { return d.sp.stages >= 2 ? spmv_tma_grid(d) : 0; }

void enqueue_spmv_tma(const DeviceLayout &d, const double *p, double *q, bool dot, cudaStream_t s) {
  SpArgs a;
  a.a_ptr = d.a_ptr;
  a.a_col = d.a_col;
  a.a_val = d.a_val;
  a.nslices = d.sp.nslices;
  a.nchunks = d.sp.nchunks;
  a.stages = d.sp.stages;
  a.off_val = d.sp.off_val;
  a.off_p = d.sp.off_p;
  a.stage_bytes = d.sp.stage_bytes;
  const unsigned grid = spmv_tma_grid(d);
  const size_t sm = (size_t)d.sp.stages * d.sp.stage_bytes;
  if (dot)
    k_spmv_tma<true><<<grid, kSpThreads, sm, s>>>(a, p, q, d.part, d.sc);
  else
    k_spmv_tma<false><<<grid, kSpThreads, sm, s>>>(a, p, q, d.part, d.sc);
}

}  // namespace hbmc

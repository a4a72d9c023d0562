// Device helpers of the warp-per-unit kernels (one warp per level-1 block),
// shared by the single-system and the batched solvers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "device_util.cuh"
#include "hbmc_internal.h"

namespace hbmc {

constexpr int kChunk = 8;

__device__ __forceinline__ int64_t rec64(const int32_t *r, int k) {
  return (int64_t)(((uint64_t)(uint32_t)r[k + 1] << 32) | (uint64_t)(uint32_t)r[k]);
}

// Deterministic sum over the CUDA block for any blockDim.x that is a
// multiple of 32 (at most 1024); valid in thread 0.
__device__ __forceinline__ double block_sum_rt(double v) {
  __shared__ double red[32];
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    s = warp_sum(s);
  }
  return s;
}

// ts[l] += sign * sum of the unit's run entries of slice l: v * src[col],
// entries taken in run order (the per-row order fixed by the layout).  The
// loads of kChunk entries are issued together before any is used.  W lanes
// per level-1 block (w = W); `lane` is the lane within the level-1 block.
template <typename T, typename G, bool kNeg, int W = 32>
__device__ __forceinline__ void run_accumulate(const int32_t *__restrict__ col, const T *__restrict__ val,
                                               const G *src, int64_t beg, int len, const int32_t *rel,
                                               T *ts, int lane) {
  int l = 0;
  for (int t0 = 0; t0 < len; t0 += kChunk * W) {
    int32_t c[kChunk];
    T v[kChunk], g[kChunk];
#pragma unroll
    for (int k = 0; k < kChunk; ++k) {
      const int t = t0 + k * W;
      if (t < len) {
        c[k] = col[beg + t + lane];
        v[k] = val[beg + t + lane];
      }
    }
#pragma unroll
    for (int k = 0; k < kChunk; ++k) {
      const int t = t0 + k * W;
      if (t < len) g[k] = (T)src[c[k]];
    }
#pragma unroll
    for (int k = 0; k < kChunk; ++k) {
      const int t = t0 + k * W;
      if (t < len) {
        while (t >= rel[l + 1]) ++l;
        T *slot = ts + l * W + lane;
        *slot = fma(kNeg ? -v[k] : v[k], g[k], *slot);
      }
    }
  }
}

// r.z of a backward sweep: this CUDA block's partial into part[slot]; in
// the sweep's last launch, the last of its `nparts` contributing blocks adds
// every partial of the sweep (part_total) in index order and takes the CG
// scalars' step (dot_mode 1: rho; 2: rho and beta).
__device__ __forceinline__ void rz_partial(double rz, Scalars *sc, int dot_mode, double *part, int64_t slot,
                                           int last_launch, int64_t part_total, unsigned nparts) {
  const double v = block_sum_rt(rz);
  if (threadIdx.x == 0) part[slot] = v;
  if (!last_launch) return;
  __shared__ unsigned s_last;
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(&sc->cnt[CNT_RZ], 1u);
    s_last = (t == nparts - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < part_total; k += blockDim.x) acc += __ldcg(part + k);
  const double rho_new = block_sum_rt(acc);
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

}  // namespace hbmc

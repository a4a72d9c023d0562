// SOR and symmetric SOR sweeps on the HBMC ordering (Section 2: the
// iteration steps of the GS and SOR methods are substitutions like those of
// IC(0); Section 3.1, Eq. "xj": an equivalent reordering gives the same
// iterates, so the colors' level-1 blocks run in parallel).
//
// One launch per color (forward sweep: colors ascending, steps ascending;
// the backward half of symmetric SOR: colors and steps descending), one CUDA
// block per level-1 block:
//   1. the level-1 block's x, b and slice offsets into shared memory;
//   2. every thread takes a share of the block's SpMV entries (Section
//      4.3.2's SELL rows of Abar, ascending columns): the coefficient, and
//      where its x value will be -- a same-block row, or the gathered x of
//      another color (earlier colors already hold this sweep's values, later
//      colors the previous ones); the diagonal gives 1 / a_ii;
//   3. lane j < w of the first warp runs BMC block j's chain of bs rows:
//      s = sum_{col != i} a_ij x_j (ascending column, fma from zero, x_j of
//      the same block from shared memory as the chain updates it),
//      t = (b_i - s) * (1 / a_ii), x_i = fma(omega, t - x_i, x_i);
//   4. the rows of x are stored.
// The operations and their order are the oracle's (orc_sor), so x is
// bit-identical to it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "device_util.cuh"
#include "hbmc_internal.h"
#include "kernels.h"

namespace hbmc {
namespace {

constexpr int kSorThreads = 256;
constexpr int kSorU = 4;
constexpr size_t kSorSmemBudget = 200 * 1024;

struct SorArgs {
  const int64_t *a_ptr;
  const int32_t *a_col;
  const double *a_val;
  int bs, w, lw;
  int64_t tile0;
  uint32_t off_cb, off_bb, off_dd, off_sv, off_ix;
};

// Shared memory of one level-1 block: rel[bs+1] slice offsets; cb = the
// block's own x (R values, updated by the chains) followed by one gathered
// x value per SpMV entry and a zero slot; bb = b; dd = 1 / a_ii; sv = the
// entries' coefficients; ix = where in cb each entry's x value lives (a
// same-block row, its own gathered slot, or the zero slot for the diagonal,
// whose coefficient then adds nothing).  Every term is then one fma with no
// branch.
template <bool FWD>
__global__ void __launch_bounds__(kSorThreads, 6)
    k_sor(const SorArgs a, double *x, const double *__restrict__ b, double omega) {
  extern __shared__ __align__(16) unsigned char smem[];
  int32_t *rel = reinterpret_cast<int32_t *>(smem);
  double *cb = reinterpret_cast<double *>(smem + a.off_cb);
  double *bb = reinterpret_cast<double *>(smem + a.off_bb);
  double *dd = reinterpret_cast<double *>(smem + a.off_dd);
  double *sv = reinterpret_cast<double *>(smem + a.off_sv);
  int32_t *ix = reinterpret_cast<int32_t *>(smem + a.off_ix);
  const int tid = threadIdx.x;
  const int64_t u = a.tile0 + blockIdx.x;
  const int R = a.bs << a.lw;
  const int64_t row0 = u * (int64_t)R, s0 = u * (int64_t)a.bs;
  const int64_t base = a.a_ptr[s0];
  const int len = (int)(a.a_ptr[s0 + a.bs] - base);
  // 1.
  for (int k = tid; k <= a.bs; k += kSorThreads) rel[k] = (int32_t)(a.a_ptr[s0 + k] - base);
  for (int lr = tid; lr < R; lr += kSorThreads) {
    cb[lr] = x[row0 + lr];
    bb[lr] = b[row0 + lr];
  }
  if (tid == 0) cb[R + len] = 0.0;
  __syncthreads();
  // 2.
  for (int e0 = tid; e0 < len; e0 += kSorThreads * kSorU) {
    int32_t c[kSorU];
    double v[kSorU], g[kSorU];
#pragma unroll
    for (int k = 0; k < kSorU; ++k) {
      const int e = e0 + k * kSorThreads;
      if (e < len) {
        c[k] = a.a_col[base + e];
        v[k] = a.a_val[base + e];
      }
    }
#pragma unroll
    for (int k = 0; k < kSorU; ++k) {
      const int e = e0 + k * kSorThreads;
      if (e < len && (c[k] < row0 || c[k] >= row0 + R)) g[k] = x[c[k]];
    }
#pragma unroll
    for (int k = 0; k < kSorU; ++k) {
      const int e = e0 + k * kSorThreads;
      if (e >= len) continue;
      sv[e] = v[k];
      if (c[k] < row0 || c[k] >= row0 + R) {
        cb[R + e] = g[k];
        ix[e] = R + e;
      } else {
        // inside the level-1 block only lane j's own BMC block couples
        const int off = (int)(c[k] - row0);
        int l = 0;
        while (e >= rel[l + 1]) ++l;  // the entry's own step
        if ((off >> a.lw) == l) {
          ix[e] = R + len;  // the diagonal: zero slot
          dd[off] = 1.0 / v[k];
        } else {
          ix[e] = off;
        }
      }
    }
  }
  __syncthreads();
  // 3.
  if (tid < a.w) {
    const int j = tid;
    for (int q = 0; q < a.bs; ++q) {
      const int l = FWD ? q : a.bs - 1 - q;
      double s = 0.0;
      const int pe = rel[l + 1];
      for (int p = rel[l] + j; p < pe; p += a.w) s = fma(sv[p], cb[ix[p]], s);
      const int lr = (l << a.lw) + j;
      // explicit roundings: no multiply-subtract contraction across t
      const double t = __dmul_rn(__dsub_rn(bb[lr], s), dd[lr]);
      cb[lr] = fma(omega, __dsub_rn(t, cb[lr]), cb[lr]);
    }
  }
  __syncthreads();
  // 4.
  for (int lr = tid; lr < R; lr += kSorThreads) x[row0 + lr] = cb[lr];
}

uint32_t a16(uint64_t v) { return (uint32_t)((v + 15) & ~uint64_t(15)); }

template <typename K>
cudaError_t allow(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSorSmemBudget);
}

}  // namespace

void plan_sor(const HostLayout &h, DeviceLayout &d) {
  SorPlan &p = d.sor;
  p = SorPlan();
  const uint64_t R = (uint64_t)h.bs * h.w, E = (uint64_t)h.max_a;
  p.off_cb = a16((uint64_t)(h.bs + 1) * 4);
  p.off_bb = a16(p.off_cb + (R + E + 1) * 8);
  p.off_dd = a16(p.off_bb + R * 8);
  p.off_sv = a16(p.off_dd + R * 8);
  p.off_ix = a16(p.off_sv + E * 8);
  const uint64_t total = a16(p.off_ix + E * 4);
  p.smem_bytes = (uint32_t)std::min<uint64_t>(total, 0xffffffffu);
  p.ok = total <= kSorSmemBudget && h.bs <= 64;
}

cudaError_t setup_sor() {
  cudaError_t e;
  if ((e = allow(k_sor<true>))) return e;
  return allow(k_sor<false>);
}

bool sor_usable(const DeviceLayout &d) { return d.sor.ok; }

void enqueue_sor(const DeviceLayout &d, double *x, const double *b, double omega, int64_t sweeps, bool symmetric,
                 cudaStream_t s) {
  SorArgs a;
  a.a_ptr = d.a_ptr;
  a.a_col = d.a_col;
  a.a_val = d.a_val;
  a.bs = d.bs;
  a.w = d.w;
  a.lw = d.lw;
  a.off_cb = d.sor.off_cb;
  a.off_bb = d.sor.off_bb;
  a.off_dd = d.sor.off_dd;
  a.off_sv = d.sor.off_sv;
  a.off_ix = d.sor.off_ix;
  for (int64_t k = 0; k < sweeps; ++k) {
    for (int c = 0; c < d.nc; ++c) {
      a.tile0 = d.tile_ptr[c];
      const unsigned grid = (unsigned)(d.tile_ptr[c + 1] - d.tile_ptr[c]);
      if (grid) k_sor<true><<<grid, kSorThreads, d.sor.smem_bytes, s>>>(a, x, b, omega);
    }
    if (!symmetric) continue;
    for (int c = d.nc - 1; c >= 0; --c) {
      a.tile0 = d.tile_ptr[c];
      const unsigned grid = (unsigned)(d.tile_ptr[c + 1] - d.tile_ptr[c]);
      if (grid) k_sor<false><<<grid, kSorThreads, d.sor.smem_bytes, s>>>(a, x, b, omega);
    }
  }
}

}  // namespace hbmc

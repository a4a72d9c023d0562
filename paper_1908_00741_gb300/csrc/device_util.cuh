// Device helpers shared by the kernel translation units: deterministic
// reductions, and thin wrappers over the sm_90+/sm_100+ PTX for mbarriers and
// TMA bulk copies.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace hbmc {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum, valid in thread 0.  FP64 arithmetic is scarce on
// this GPU (about 2 FP64 operations per clock per SM), so the tree is built
// to issue few FP64 warp instructions: every thread parks its value in
// shared memory, one warp adds NT/32 values per lane, then a 5-step
// butterfly finishes (NT/32 - 1 + 5 FP64 warp instructions per block).
template <int NT>
__device__ double block_sum(double v) {
  __shared__ double red[NT];
  __syncthreads();
  red[threadIdx.x] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = red[threadIdx.x];
#pragma unroll
    for (int k = 1; k < NT / 32; ++k) s += red[threadIdx.x + 32 * k];
    s = warp_sum(s);
  }
  return s;
}

// Thread 0 stores the block's partial(s); returns true in every thread of
// the last block of the grid to arrive.
__device__ __forceinline__ bool publish(double *slot, const double *vals, int nv, unsigned *cnt, unsigned nblocks) {
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
// Conversions between binary32 and binary64 with integer operations.  On this
// GPU a float <-> double conversion instruction issues on the FP64 pipe,
// which retires about two operations per clock per SM, as slowly as an FP64
// fused multiply-add.  The bulk-copy warp sweeps (sweep_tw.cu) convert every
// row they read or write in FP32, and every warp of a color's single wave
// converts at the same moment, so there the conversions queue on that pipe.
// These do the same conversions from the IEEE-754 interchange formats (sign,
// biased exponent, significand) on the integer pipe, with the same results:
// widening is exact, narrowing rounds to nearest with ties to even, as the
// casts do.  Checked against the casts by hbmc_debug_convert's test.  Where
// the FP64 pipe is not the queue (the other sweep kernels, the batched
// solver) their dozen integer instructions cost more than the cast, and the
// casts stay.
// ---------------------------------------------------------------------------

// float -> double, exact.  Normal numbers move their significand 29 bits up
// and rebias the exponent (1023 - 127 = 896); subnormal floats (m * 2^-149)
// become normal doubles; zeros, infinities and NaNs keep their class.
__device__ __forceinline__ double widen_f32(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
  const uint32_t a = u & 0x7fffffffu;
  uint64_t r = ((uint64_t)a << 29) + (896ull << 52);
  if (a - 0x00800000u >= 0x7f000000u) {  // not a normal number
    if (a == 0) {
      r = 0;
    } else if (a >= 0x7f800000u) {
      r = 0x7ff0000000000000ull | ((uint64_t)(a & 0x007fffffu) << 29);
    } else {  // subnormal: a * 2^-149 with its leading one at bit k
      const int k = 31 - __clz(a);
      r = ((uint64_t)(k + 874) << 52) | (((uint64_t)a << (52 - k)) & 0x000fffffffffffffull);
    }
  }
  return __longlong_as_double((long long)(r | sign));
}

// double -> float, rounding to nearest, ties to even.  In the float normal
// range the top 35 bits of the magnitude hold the float's exponent and
// significand (rebiased by 896); the 29 bits below decide the rounding, and
// a carry out of the significand steps the exponent (to infinity past the
// largest float).  Results in the float subnormal range round m * 2^-149;
// overflow gives infinity, and NaNs stay NaN.
__device__ __forceinline__ float narrow_f64(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const uint64_t a = b & 0x7fffffffffffffffull;
  uint32_t r;
  if (a - (897ull << 52) < (254ull << 52)) {  // 2^-126 <= |x| < 2^128
    const uint64_t t = a >> 29;
    const uint32_t rem = (uint32_t)a & 0x1fffffffu;
    const uint64_t up = (rem > 0x10000000u || (rem == 0x10000000u && (t & 1))) ? 1 : 0;
    r = (uint32_t)(t + up - (896ull << 23));
  } else if (a >= 0x7ff0000000000000ull) {  // infinity or NaN
    r = a == 0x7ff0000000000000ull ? 0x7f800000u : 0x7fffffffu;
  } else if (a >= (1151ull << 52)) {  // beyond the float range
    r = 0x7f800000u;
  } else {  // below 2^-126: the nearest multiple of 2^-149 (doubles below 2^-1022 give 0)
    const int e = (int)(a >> 52);
    const int shift = 926 - e;  // m = significand * 2^-shift
    r = 0;
    if (e > 0 && shift < 64) {
      const uint64_t mant = (a & 0x000fffffffffffffull) | (1ull << 52);
      const uint64_t kept = mant >> shift;
      const uint64_t rem = mant & ((1ull << shift) - 1);
      const uint64_t half = 1ull << (shift - 1);
      r = (uint32_t)(kept + ((rem > half || (rem == half && (kept & 1))) ? 1 : 0));
    }
  }
  return __uint_as_float(sign | r);
}

// Value conversion between the substitutions' types without the FP64 pipe.
template <typename TO, typename FROM>
__device__ __forceinline__ TO cvt(FROM v) {
  if constexpr (sizeof(TO) == sizeof(FROM)) return (TO)v;
  else if constexpr (sizeof(TO) == 8) return widen_f32(v);
  else return narrow_f64(v);
}

// Backward sweeps in FP32 gather z from its FP32 copy z32: z holds those
// FP32 results widened, so the narrowed gather gives the same value at half
// the bytes and without an FP64-pipe conversion.  FP64 sweeps gather z.
template <typename T>
__device__ __forceinline__ const T *zgather(const double *z, const float *z32) {
  if constexpr (sizeof(T) == 4) return reinterpret_cast<const T *>(z32);
  else return reinterpret_cast<const T *>(z);
}

// Row `row` of the variable-slice-height SpMV layout (hbmc_options.sell_vslice):
// row j of slice s lies in sub-slice vs_first[s] + j / C (C = vs_c[s], a
// power of two) at position j % C, its entry t at vs_ptr[sub] + t * C +
// position; summed from zero in ascending column order with one fused
// multiply-add per term, as every SpMV of the library sums a row.
__device__ __forceinline__ double vs_row(const uint8_t *__restrict__ vs_c, const int64_t *__restrict__ vs_first,
                                         const int64_t *__restrict__ vs_ptr, const int32_t *__restrict__ col,
                                         const double *__restrict__ val, int w, int lw, int64_t row,
                                         const double *x) {
  const int64_t s = row >> lw;
  const int j = (int)(row & (w - 1));
  const int C = vs_c[s];
  const int64_t sub = vs_first[s] + j / C;
  const int64_t e = vs_ptr[sub + 1];
  double acc = 0.0;
  for (int64_t q = vs_ptr[sub] + (j & (C - 1)); q < e; q += C) acc = fma(val[q], __ldg(x + col[q]), acc);
  return acc;
}

// Row kernels run a fixed grid (a few CUDA blocks per SM) and loop over the
// rows with a grid stride, so each thread accumulates its dot-product terms
// over several rows before the block reduction.
#define FOR_ROWS(row, n) \
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < (n); row += (int64_t)gridDim.x * blockDim.x)

// ---------------------------------------------------------------------------
// mbarrier / TMA bulk copy (PTX ISA 8.0+, sm_90 and later)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes barrier initialisation visible to the other threads and to the TMA unit.
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Raises the barrier's expected transaction bytes without arriving.
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for the given phase parity: false once `deadline_ns` of the
// global timer has passed without the phase completing.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t deadline_ns) {
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() > deadline_ns) return false;
  }
  return true;
}

// Orders this thread's earlier generic-proxy accesses of shared memory
// before later async-proxy (bulk copy) accesses of it.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 1-D bulk copy global -> shared memory of this CTA, completing on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Completion flags of the dependency-driven sweeps: a release store by the
// producing CUDA block after its rows are written, acquire loads by the
// consumers before they gather those rows.
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned ld_relaxed_gpu(const unsigned *p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed_gpu(unsigned *p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bulk prefetch of global memory into L2 (no completion to wait for).
// src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void prefetch_l2(const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Named barrier over `count` threads (a multiple of 32).
__device__ __forceinline__ void named_sync(uint32_t id, uint32_t count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

}  // namespace hbmc

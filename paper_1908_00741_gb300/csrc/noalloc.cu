// hbmc_spmv_dot_static: q = Abar p and p.q with no allocation at all.
//
// Some callers cannot allocate device memory at the moment they need the
// product: programs whose device memory is entirely owned by another
// allocator (for instance a framework's caching allocator with a fixed
// budget, where a cudaMalloc of our own could fail or fragment its pool),
// and latency-critical loops that forbid allocation after start-up
// (cudaMalloc may synchronize the device).  This entry point serves them.  It is the
// warp-per-level-1-block SpMV with the fused p.q of the solver, except that
// its reduction scratch (one partial sum per CUDA block and an arrival
// counter) lives in a fixed-size array in the library's own static device
// memory instead of memory a context allocates.
//
// The array is file-scope and shared by every call on a device; it keeps the
// last call's contents.  Each call clears the counter on its stream before
// launching, but two calls whose kernels overlap on the GPU (different
// streams, no ordering between them) would race on the array: order them.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>

#include "hbmc.h"
#include "hbmc_internal.h"

namespace hbmc {
bool ctx_view(hbmc_ctx *ctx, const DeviceLayout **d, cudaStream_t *stream, int *device,
              bool *factored, std::string **err);
}

namespace {

using hbmc::DeviceLayout;

// At most this many CUDA blocks of 4 warps, i.e. 4 * 8192 = 32768 level-1
// blocks (8,388,608 rows at bs = 8, w = 32).  Layout: 16 bytes holding the
// arrival counter, then one double per CUDA block.
constexpr int kStaticBlocks = 8192;
constexpr int kWarps = 4;
constexpr int kMaxDevices = 64;
static __device__ __align__(256) unsigned char g_spmv_scratch[16 + kStaticBlocks * sizeof(double)];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

__device__ __forceinline__ double sum_warp(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum in a fixed order, valid in thread 0.
__device__ double sum_block(double v) {
  __shared__ double red[kWarps];
  v = sum_warp(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    s = sum_warp(s);
  }
  return s;
}

// One warp per level-1 block: each lane accumulates its bs rows over the
// block's run of entries (ascending column inside every row, one fused
// multiply-add per entry, from zero), so q matches hbmc_spmv_bar bit for
// bit.  Padded slots (column n_pad) read as 0 instead of a guard entry,
// because the caller's vector has exactly n_pad entries.
__global__ void __launch_bounds__(32 * kWarps)
    k_spmv_dot_static(const int32_t *__restrict__ rec, int rec_ints, const int32_t *__restrict__ a_col,
                      const double *__restrict__ a_val, int bs, int64_t units, int64_t n_pad,
                      const double *__restrict__ p, double *__restrict__ q, double *pq_out,
                      unsigned char *scratch) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t u = (int64_t)blockIdx.x * kWarps + warp;
  const size_t rec_bytes = ((size_t)rec_ints * 4 + 15) & ~size_t(15);
  const size_t warp_bytes = rec_bytes + (size_t)bs * 32 * sizeof(double);
  int32_t *rs = reinterpret_cast<int32_t *>(smem + warp * warp_bytes);
  double *ts = reinterpret_cast<double *>(smem + warp * warp_bytes + rec_bytes);
  double pq = 0.0;
  if (u < units) {
    for (int k = lane; k < rec_ints; k += 32) rs[k] = rec[u * rec_ints + k];
    for (int l = 0; l < bs; ++l) ts[(l << 5) + lane] = 0.0;
    __syncwarp();
    const int len = rs[0];
    const int64_t beg = (int64_t)(((uint64_t)(uint32_t)rs[3] << 32) | (uint64_t)(uint32_t)rs[2]);
    const int32_t *rel = rs + 6;
    int l = 0;
    for (int t = 0; t < len; t += 32) {
      while (t >= rel[l + 1]) ++l;
      const int32_t c = a_col[beg + t + lane];
      const double g = c < n_pad ? p[c] : 0.0;
      ts[(l << 5) + lane] = fma(a_val[beg + t + lane], g, ts[(l << 5) + lane]);
    }
    const int64_t row0 = u * (int64_t)bs * 32;
    for (int k = 0; k < bs; ++k) {
      const double qv = ts[(k << 5) + lane];
      q[row0 + (k << 5) + lane] = qv;
      pq = fma(p[row0 + (k << 5) + lane], qv, pq);
    }
  }
  unsigned int *counter = reinterpret_cast<unsigned int *>(scratch);
  double *partial = reinterpret_cast<double *>(scratch + 16);
  const double v = sum_block(pq);
  __shared__ unsigned int last;
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = v;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < gridDim.x; k += blockDim.x) acc += __ldcg(partial + k);
  const double s = sum_block(acc);
  if (threadIdx.x == 0) {
    *pq_out = s;
    *counter = 0;
  }
}

// Once per device, with that device current: the device address of the
// static array (its host-side name is only a stand-in and must never reach a
// kernel) and the kernel's shared-memory limit.
hbmc_status scratch_for_device(int dev, unsigned char **out, std::string &err) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (dev < 0 || dev >= kMaxDevices) {
    err = "hbmc_spmv_dot_static: device ordinal out of range";
    return HBMC_ERR_INVALID_ARG;
  }
  if (!g_scratch_ptr[dev]) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_spmv_scratch);
    if (e != cudaSuccess) {
      err = std::string("hbmc_spmv_dot_static: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
      return HBMC_ERR_CUDA;
    }
    e = cudaFuncSetAttribute(k_spmv_dot_static, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kWarps * (16 * 1024 + 2 * 1024));
    if (e != cudaSuccess) {
      err = std::string("hbmc_spmv_dot_static: cudaFuncSetAttribute failed: ") + cudaGetErrorString(e);
      return HBMC_ERR_CUDA;
    }
    g_scratch_ptr[dev] = ptr;
  }
  *out = static_cast<unsigned char *>(g_scratch_ptr[dev]);
  return HBMC_OK;
}

}  // namespace

extern "C" hbmc_status hbmc_spmv_dot_static(hbmc_ctx *ctx, const double *p_dev, double *q_dev,
                                            double *pq_dev) {
  const DeviceLayout *d = nullptr;
  cudaStream_t stream = nullptr;
  int dev = 0;
  bool factored = false;
  std::string *err = nullptr;
  if (!hbmc::ctx_view(ctx, &d, &stream, &dev, &factored, &err)) return HBMC_ERR_NO_DEVICE;
  if (d->n == 0) {
    // nothing to multiply; p.q of empty vectors is 0, written so that the
    // caller never reads a stale value after a successful call
    if (!pq_dev) {
      *err = "hbmc_spmv_dot_static: null pointer";
      return HBMC_ERR_INVALID_ARG;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
    const cudaError_t e = cudaMemsetAsync(pq_dev, 0, sizeof(double), stream);
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    if (e != cudaSuccess) {
      *err = std::string("hbmc_spmv_dot_static: ") + cudaGetErrorString(e);
      return HBMC_ERR_CUDA;
    }
    return HBMC_OK;
  }
  if (!p_dev || !q_dev || !pq_dev) {
    *err = "hbmc_spmv_dot_static: null pointer";
    return HBMC_ERR_INVALID_ARG;
  }
  if (d->w != 32 || !d->rec_a) {
    *err = "hbmc_spmv_dot_static: needs a context built with w = 32";
    return HBMC_ERR_INVALID_ARG;
  }
  const int64_t units = d->tile_ptr[d->nc];
  const int64_t blocks = (units + kWarps - 1) / kWarps;
  if (blocks > kStaticBlocks) {
    char buf[200];
    std::snprintf(buf, sizeof buf,
                  "hbmc_spmv_dot_static: %lld level-1 blocks exceed the static scratch limit of %d "
                  "(n_pad %lld > %lld rows at bs = %d)",
                  (long long)units, kStaticBlocks * kWarps, (long long)d->n_pad,
                  (long long)kStaticBlocks * kWarps * d->bs * 32, d->bs);
    *err = buf;
    return HBMC_ERR_INVALID_ARG;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != dev) cudaSetDevice(dev);
  unsigned char *scratch = nullptr;
  hbmc_status st = scratch_for_device(dev, &scratch, *err);
  if (st == HBMC_OK) {
    cudaError_t e = cudaMemsetAsync(scratch, 0, 16, stream);
    if (e == cudaSuccess) {
      const size_t rec_bytes = ((size_t)d->rec_ints * 4 + 15) & ~size_t(15);
      const size_t smem = kWarps * (rec_bytes + (size_t)d->bs * 32 * sizeof(double));
      k_spmv_dot_static<<<(unsigned)blocks, 32 * kWarps, smem, stream>>>(
          d->rec_a, d->rec_ints, d->a_col, d->a_val, d->bs, units, d->n_pad, p_dev, q_dev, pq_dev, scratch);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
      *err = std::string("hbmc_spmv_dot_static: ") + cudaGetErrorString(e);
      st = HBMC_ERR_CUDA;
    }
  }
  if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  return st;
}

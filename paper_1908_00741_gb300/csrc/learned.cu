// Learned IC(0) shift: matrix features, a small MLP (forward, backward, Adam)
// and shift selection with the plain positive-pivot rule as fallback.
//
// The paper's shifted ICCG (Section 5.1) fixes the shift by hand (0.3 for
// the Ieej system).  Here a network predicts, from cheap matrix features and
// a candidate shift, how many CG iterations that shift would cost; the
// candidate with the lowest prediction is tried first.  If its IC(0) meets a
// pivot that is not positive, the plain rule takes over: shift 0, then
// 1e-3 * 2^k (k = 0, 1, ...) until every pivot is positive.
//
// Everything numeric runs in these kernels: the feature reduction over the
// matrix (one warp per level-1 block, then one CUDA block per system), the
// network's forward pass (one warp per sample, lane = hidden unit), the
// per-sample gradients, their reduction in a fixed order, and Adam.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "device_util.cuh"
#include "hbmc.h"
#include "hbmc_internal.h"
#include "warp_common.cuh"

namespace hbmc {
namespace {

constexpr int kFeat = HBMC_NUM_FEATURES;  // 12
constexpr int kPart = 11;                 // per-unit partial statistics
constexpr int kH = 32;                    // hidden width = one warp
constexpr double kDomCap = 10.0;
// rows count as weakly dominated below 1 - 1e-9 (exactly balanced rows such as
// interior stencil rows sit at 1 up to rounding and must not flip)
constexpr double kWeak = 1.0 - 1e-9;

// ---------------------------------------------------------------------------
// features
// ---------------------------------------------------------------------------
// Per-unit partials over the unit's real (non-dummy) rows of Abar:
//  0 rows, 1 sum nnz, 2 max nnz, 3 min dominance, 4 sum dominance,
//  5 rows with dominance < 1 - 1e-9, 6 positive off-diagonals, 7 off-diagonals,
//  8 sum log a_ii, 9 sum (log a_ii)^2, 10 max dominance
// where dominance = a_ii / sum_{j != i} |a_ij| (capped at kDomCap).
__global__ void __launch_bounds__(128)
    k_feat_units(const int32_t *__restrict__ rec, int rec_ints, const int32_t *__restrict__ a_col,
                 const double *__restrict__ a_val, const double *__restrict__ adiag, const int32_t *__restrict__ inv,
                 int bs, int64_t units, int64_t n_pad, double *part) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t u = (int64_t)blockIdx.x * 4 + warp;
  if (u >= units) return;
  const int32_t *rc = rec + u * rec_ints;
  const int64_t beg = rec64(rc, 2);
  double rows = 0, nnz = 0, maxnnz = 0, mindom = kDomCap, sumdom = 0, weak = 0, pos = 0, off = 0, sl = 0, sl2 = 0,
         maxdom = 0;
  for (int l = 0; l < bs; ++l) {
    const int64_t row = (u * bs + l) * 32 + lane;
    if (inv[row] < 0) continue;
    const double d = adiag[row];
    double offsum = 0.0, cnt = 0.0, npos = 0.0;
    for (int p = rc[6 + l] + lane; p < rc[7 + l]; p += 32) {
      const int32_t c = a_col[beg + p];
      if (c >= n_pad) continue;  // slice padding
      cnt += 1.0;
      if (c == row) continue;
      const double v = a_val[beg + p];
      offsum += fabs(v);
      if (v > 0.0) npos += 1.0;
    }
    const double dom = offsum > 0.0 ? fmin(d / offsum, kDomCap) : kDomCap;
    rows += 1.0;
    nnz += cnt;
    maxnnz = fmax(maxnnz, cnt);
    mindom = fmin(mindom, dom);
    maxdom = fmax(maxdom, dom);
    sumdom += dom;
    if (dom < kWeak) weak += 1.0;
    pos += npos;
    off += cnt - 1.0;
    const double lg = log(d);
    sl += lg;
    sl2 += lg * lg;
  }
  double v[kPart] = {rows, nnz, maxnnz, mindom, sumdom, weak, pos, off, sl, sl2, maxdom};
#pragma unroll
  for (int k = 0; k < kPart; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_xor_sync(0xffffffffu, v[k], o);
      v[k] = (k == 2 || k == 10) ? fmax(v[k], w) : (k == 3 ? fmin(v[k], w) : v[k] + w);
    }
  }
  if (lane == 0)
    for (int k = 0; k < kPart; ++k) part[u * kPart + k] = v[k];
}

// One CUDA block per system: combine its units' partials (fixed order) into
// the feature vector.
__global__ void __launch_bounds__(256)
    k_feat_finish(int32_t nc, const int64_t *__restrict__ cu_start, const int64_t *__restrict__ cu_count,
                  const double *part, const int32_t *__restrict__ nc_sys, int bs, float *feat) {
  const int s = blockIdx.x;
  __shared__ double acc[256][kPart];
  double v[kPart] = {0, 0, 0, kDomCap, 0, 0, 0, 0, 0, 0, 0};
  for (int c = 0; c < nc; ++c) {
    const int64_t u0 = cu_start[(int64_t)s * nc + c], cnt = cu_count[(int64_t)s * nc + c];
    for (int64_t k = threadIdx.x; k < cnt; k += 256) {
      const double *p = part + (u0 + k) * kPart;
      for (int q = 0; q < kPart; ++q)
        v[q] = (q == 2 || q == 10) ? fmax(v[q], p[q]) : (q == 3 ? fmin(v[q], p[q]) : v[q] + p[q]);
    }
  }
  for (int q = 0; q < kPart; ++q) acc[threadIdx.x][q] = v[q];
  __syncthreads();
  if (threadIdx.x != 0) return;
  double t[kPart];
  for (int q = 0; q < kPart; ++q) t[q] = acc[0][q];
  for (int k = 1; k < 256; ++k)
    for (int q = 0; q < kPart; ++q)
      t[q] = (q == 2 || q == 10) ? fmax(t[q], acc[k][q]) : (q == 3 ? fmin(t[q], acc[k][q]) : t[q] + acc[k][q]);
  const double rows = fmax(t[0], 1.0);
  const double mean_l = t[8] / rows;
  float *f = feat + (int64_t)s * kFeat;
  f[0] = (float)log10(rows);
  f[1] = (float)(t[1] / rows);
  f[2] = (float)t[2];
  f[3] = (float)t[3];
  f[4] = (float)(t[4] / rows);
  f[5] = (float)(t[5] / rows);
  f[6] = (float)(t[7] > 0 ? t[6] / t[7] : 0.0);
  f[7] = (float)mean_l;
  f[8] = (float)sqrt(fmax(t[9] / rows - mean_l * mean_l, 0.0));
  f[9] = (float)(nc_sys ? nc_sys[s] : nc);
  f[10] = (float)bs;
  f[11] = (float)t[10];
}

// ---------------------------------------------------------------------------
// MLP  D -> 32 -> 32 -> 1, ReLU; inputs standardized with (mean, std)
// Parameter layout: W1[H][D], b1[H], W2[H][H], b2[H], w3[H], b3
// ---------------------------------------------------------------------------
struct MlpDev {
  int D;
  const float *p;      // parameters
  const float *mean;   // D
  const float *stdv;   // D
};

__device__ __forceinline__ int off_b1(int D) { return kH * D; }
__device__ __forceinline__ int off_W2(int D) { return kH * D + kH; }
__device__ __forceinline__ int off_b2(int D) { return kH * D + kH + kH * kH; }
__device__ __forceinline__ int off_w3(int D) { return kH * D + 2 * kH + kH * kH; }
__device__ __forceinline__ int off_b3(int D) { return kH * D + 3 * kH + kH * kH; }

// one warp per sample; lane = hidden unit h
__global__ void __launch_bounds__(128)
    k_mlp_forward(MlpDev m, const float *__restrict__ X, int B, float *out, float *z1s, float *z2s) {
  const int warp = threadIdx.x >> 5, h = threadIdx.x & 31;
  const int b = blockIdx.x * 4 + warp;
  if (b >= B) return;
  const int D = m.D;
  const float *x = X + (int64_t)b * D;
  float z1 = m.p[off_b1(D) + h];
  for (int d = 0; d < D; ++d) z1 = fmaf(m.p[h * D + d], (x[d] - m.mean[d]) / m.stdv[d], z1);
  const float a1 = fmaxf(z1, 0.f);
  float z2 = m.p[off_b2(D) + h];
  for (int k = 0; k < kH; ++k) z2 = fmaf(m.p[off_W2(D) + h * kH + k], __shfl_sync(0xffffffffu, a1, k), z2);
  const float a2 = fmaxf(z2, 0.f);
  float o = m.p[off_w3(D) + h] * a2;
  for (int s = 16; s > 0; s >>= 1) o += __shfl_xor_sync(0xffffffffu, o, s);
  if (z1s) z1s[(int64_t)b * kH + h] = z1;
  if (z2s) z2s[(int64_t)b * kH + h] = z2;
  if (h == 0) out[b] = o + m.p[off_b3(D)];
}

// Per-sample gradient of L = (1/B) sum_b (out_b - t_b)^2 into G[b][P].
__global__ void __launch_bounds__(128)
    k_mlp_sample_grad(MlpDev m, const float *__restrict__ X, const float *__restrict__ T, const float *out,
                      const float *z1s, const float *z2s, int B, int P, float *G) {
  const int warp = threadIdx.x >> 5, h = threadIdx.x & 31;
  const int b = blockIdx.x * 4 + warp;
  if (b >= B) return;
  const int D = m.D;
  const float *x = X + (int64_t)b * D;
  float *g = G + (int64_t)b * P;
  const float z1 = z1s[(int64_t)b * kH + h], z2 = z2s[(int64_t)b * kH + h];
  const float a1 = fmaxf(z1, 0.f), a2 = fmaxf(z2, 0.f);
  const float dout = 2.f * (out[b] - T[b]) / (float)B;
  g[off_w3(D) + h] = dout * a2;
  if (h == 0) g[off_b3(D)] = dout;
  const float dz2 = z2 > 0.f ? dout * m.p[off_w3(D) + h] : 0.f;
  g[off_b2(D) + h] = dz2;
  for (int k = 0; k < kH; ++k) g[off_W2(D) + h * kH + k] = dz2 * __shfl_sync(0xffffffffu, a1, k);
  // da1[h] = sum_j W2[j][h] dz2[j]
  float da1 = 0.f;
  for (int j = 0; j < kH; ++j) da1 = fmaf(m.p[off_W2(D) + j * kH + h], __shfl_sync(0xffffffffu, dz2, j), da1);
  const float dz1 = z1 > 0.f ? da1 : 0.f;
  g[off_b1(D) + h] = dz1;
  for (int d = 0; d < D; ++d) g[h * D + d] = dz1 * ((x[d] - m.mean[d]) / m.stdv[d]);
}

// grad[p] = sum_b G[b][p] in sample order; loss = sum_b (out_b - t_b)^2 / B
__global__ void k_mlp_reduce(const float *G, int B, int P, float *grad, const float *out, const float *T,
                             float *loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < P) {
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += G[(int64_t)b * P + p];
    grad[p] = s;
  }
  if (p == 0 && loss) {
    float l = 0.f;
    for (int b = 0; b < B; ++b) l += (out[b] - T[b]) * (out[b] - T[b]);
    *loss = l / (float)B;
  }
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, int P, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  m[i] = b1 * m[i] + (1.f - b1) * g[i];
  v[i] = b2 * v[i] + (1.f - b2) * g[i] * g[i];
  p[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
}

// candidate inputs: features of one system followed by shift code c/(ncand-1)
__global__ void k_candidates(const float *feat, int ncand, float *X) {
  const int c = threadIdx.x;
  if (c >= ncand) return;
  for (int k = 0; k < kFeat; ++k) X[c * (kFeat + 1) + k] = feat[k];
  X[c * (kFeat + 1) + kFeat] = (float)c / (float)(ncand - 1);
}

unsigned nb(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// Features of a device layout viewed as `nsys` systems (unit_sys == nullptr:
// one system).  Host buffers for the per-system unit ranges are uploaded
// temporarily; feat_dev receives nsys * HBMC_NUM_FEATURES floats.
hbmc_status features_on_device(const DeviceLayout &d, int32_t nsys, const int64_t *cu_start_dev,
                               const int64_t *cu_count_dev, const int32_t *nc_sys_dev, float *feat_dev,
                               cudaStream_t s, std::string &err) {
  const int64_t units = d.tile_ptr[d.nc];
  double *part = nullptr;
  int64_t *cs = nullptr, *cc = nullptr;
  cudaError_t e = cudaMallocAsync(&part, sizeof(double) * kPart * (units ? units : 1), s);
  std::vector<int64_t> hs, hc;
  if (e == cudaSuccess && !cu_start_dev) {
    hs.resize(d.nc);
    hc.resize(d.nc);
    for (int c = 0; c < d.nc; ++c) {
      hs[c] = d.tile_ptr[c];
      hc[c] = d.tile_ptr[c + 1] - d.tile_ptr[c];
    }
    e = cudaMallocAsync(&cs, sizeof(int64_t) * (d.nc ? d.nc : 1), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&cc, sizeof(int64_t) * (d.nc ? d.nc : 1), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cs, hs.data(), sizeof(int64_t) * d.nc, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cc, hc.data(), sizeof(int64_t) * d.nc, cudaMemcpyHostToDevice, s);
    cu_start_dev = cs;
    cu_count_dev = cc;
  }
  if (e == cudaSuccess && units > 0) {
    k_feat_units<<<nb(units, 4), 128, 0, s>>>(d.rec_a, d.rec_ints, d.a_col, d.a_val, d.adiag, d.inv, d.bs, units,
                                             d.n_pad, part);
    k_feat_finish<<<nsys, 256, 0, s>>>(d.nc, cu_start_dev, cu_count_dev, part, nc_sys_dev, d.bs, feat_dev);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (part) cudaFreeAsync(part, s);
  if (cs) cudaFreeAsync(cs, s);
  if (cc) cudaFreeAsync(cc, s);
  cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    err = std::string("features: ") + cudaGetErrorString(e);
    return HBMC_ERR_CUDA;
  }
  return HBMC_OK;
}

}  // namespace hbmc

// ===========================================================================
// MLP handle and C ABI
// ===========================================================================
struct hbmc_mlp {
  int D = 0, P = 0, cap = 0;
  float *p = nullptr, *mean = nullptr, *stdv = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  float *out = nullptr, *z1 = nullptr, *z2 = nullptr, *G = nullptr, *loss = nullptr;
  int64_t step = 0;
  std::string err;
};

namespace {

thread_local std::string g_mlp_err;

hbmc::MlpDev mlp_view(const hbmc_mlp *n) {
  hbmc::MlpDev m;
  m.D = n->D;
  m.p = n->p;
  m.mean = n->mean;
  m.stdv = n->stdv;
  return m;
}

hbmc_status ensure_cap(hbmc_mlp *n, int B) {
  if (B <= n->cap) return HBMC_OK;
  cudaFree(n->out);
  cudaFree(n->z1);
  cudaFree(n->z2);
  cudaFree(n->G);
  n->out = n->z1 = n->z2 = n->G = nullptr;
  n->cap = 0;
  if (cudaMalloc(&n->out, sizeof(float) * B) != cudaSuccess ||
      cudaMalloc(&n->z1, sizeof(float) * (int64_t)B * hbmc::kH) != cudaSuccess ||
      cudaMalloc(&n->z2, sizeof(float) * (int64_t)B * hbmc::kH) != cudaSuccess ||
      cudaMalloc(&n->G, sizeof(float) * (int64_t)B * n->P) != cudaSuccess) {
    n->err = "mlp: out of device memory";
    return HBMC_ERR_OOM;
  }
  n->cap = B;
  return HBMC_OK;
}

hbmc_status mlp_grad(hbmc_mlp *n, const float *X, const float *T, int B, float *grad, float *loss_dev) {
  hbmc_status s = ensure_cap(n, B);
  if (s != HBMC_OK) return s;
  hbmc::k_mlp_forward<<<hbmc::nb(B, 4), 128>>>(mlp_view(n), X, B, n->out, n->z1, n->z2);
  hbmc::k_mlp_sample_grad<<<hbmc::nb(B, 4), 128>>>(mlp_view(n), X, T, n->out, n->z1, n->z2, B, n->P, n->G);
  hbmc::k_mlp_reduce<<<hbmc::nb(n->P, 256), 256>>>(n->G, B, n->P, grad, n->out, T, loss_dev);
  if (cudaGetLastError() != cudaSuccess) {
    n->err = "mlp: kernel launch failed";
    return HBMC_ERR_CUDA;
  }
  return HBMC_OK;
}

const double kShiftGrid0 = 1e-3;

double grid_shift(int c) { return c == 0 ? 0.0 : kShiftGrid0 * std::ldexp(1.0, c - 1); }

}  // namespace

extern "C" {

int32_t hbmc_mlp_num_params(int32_t in_dim) { return hbmc::kH * in_dim + 3 * hbmc::kH + hbmc::kH * hbmc::kH + 1; }

hbmc_status hbmc_mlp_create(int32_t in_dim, hbmc_mlp **out) {
  if (!out || in_dim < 1 || in_dim > 256) {
    g_mlp_err = "mlp: in_dim must be in [1, 256]";
    return HBMC_ERR_INVALID_ARG;
  }
  *out = nullptr;
  hbmc_mlp *n = new hbmc_mlp();
  n->D = in_dim;
  n->P = hbmc_mlp_num_params(in_dim);
  if (cudaMalloc(&n->p, sizeof(float) * n->P) != cudaSuccess ||
      cudaMalloc(&n->grad, sizeof(float) * n->P) != cudaSuccess ||
      cudaMalloc(&n->m, sizeof(float) * n->P) != cudaSuccess ||
      cudaMalloc(&n->v, sizeof(float) * n->P) != cudaSuccess ||
      cudaMalloc(&n->mean, sizeof(float) * in_dim) != cudaSuccess ||
      cudaMalloc(&n->stdv, sizeof(float) * in_dim) != cudaSuccess ||
      cudaMalloc(&n->loss, sizeof(float)) != cudaSuccess) {
    g_mlp_err = "mlp: out of device memory";
    hbmc_mlp_destroy(n);
    return HBMC_ERR_OOM;
  }
  cudaMemset(n->p, 0, sizeof(float) * n->P);
  cudaMemset(n->m, 0, sizeof(float) * n->P);
  cudaMemset(n->v, 0, sizeof(float) * n->P);
  cudaMemset(n->mean, 0, sizeof(float) * in_dim);
  std::vector<float> ones(in_dim, 1.f);
  cudaMemcpy(n->stdv, ones.data(), sizeof(float) * in_dim, cudaMemcpyHostToDevice);
  *out = n;
  return HBMC_OK;
}

void hbmc_mlp_destroy(hbmc_mlp *n) {
  if (!n) return;
  for (float *q : {n->p, n->mean, n->stdv, n->grad, n->m, n->v, n->out, n->z1, n->z2, n->G, n->loss}) cudaFree(q);
  delete n;
}

const char *hbmc_mlp_last_error(const hbmc_mlp *n) { return n ? n->err.c_str() : g_mlp_err.c_str(); }

hbmc_status hbmc_mlp_set_params(hbmc_mlp *n, const float *params, const float *in_mean, const float *in_std) {
  if (!n) return HBMC_ERR_INVALID_ARG;
  if (params && cudaMemcpy(n->p, params, sizeof(float) * n->P, cudaMemcpyHostToDevice) != cudaSuccess)
    return HBMC_ERR_CUDA;
  if (in_mean && cudaMemcpy(n->mean, in_mean, sizeof(float) * n->D, cudaMemcpyHostToDevice) != cudaSuccess)
    return HBMC_ERR_CUDA;
  if (in_std) {
    for (int d = 0; d < n->D; ++d)
      if (!(in_std[d] > 0.f)) {
        n->err = "mlp: input std must be positive";
        return HBMC_ERR_INVALID_ARG;
      }
    if (cudaMemcpy(n->stdv, in_std, sizeof(float) * n->D, cudaMemcpyHostToDevice) != cudaSuccess)
      return HBMC_ERR_CUDA;
  }
  cudaMemset(n->m, 0, sizeof(float) * n->P);
  cudaMemset(n->v, 0, sizeof(float) * n->P);
  n->step = 0;
  return HBMC_OK;
}

hbmc_status hbmc_mlp_get_params(const hbmc_mlp *n, float *params) {
  if (!n || !params) return HBMC_ERR_INVALID_ARG;
  return cudaMemcpy(params, n->p, sizeof(float) * n->P, cudaMemcpyDeviceToHost) == cudaSuccess ? HBMC_OK
                                                                                                 : HBMC_ERR_CUDA;
}

hbmc_status hbmc_mlp_forward(hbmc_mlp *n, const float *X_dev, int32_t B, float *out_dev) {
  if (!n || !X_dev || !out_dev || B < 0) return HBMC_ERR_INVALID_ARG;
  if (B == 0) return HBMC_OK;
  hbmc::k_mlp_forward<<<hbmc::nb(B, 4), 128>>>(mlp_view(n), X_dev, B, out_dev, nullptr, nullptr);
  if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return HBMC_ERR_CUDA;
  return HBMC_OK;
}

hbmc_status hbmc_mlp_gradient(hbmc_mlp *n, const float *X_dev, const float *T_dev, int32_t B, float *grad_dev,
                              float *loss) {
  if (!n || !X_dev || !T_dev || !grad_dev || B < 1) return HBMC_ERR_INVALID_ARG;
  hbmc_status s = mlp_grad(n, X_dev, T_dev, B, grad_dev, n->loss);
  if (s != HBMC_OK) return s;
  if (loss && cudaMemcpy(loss, n->loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return HBMC_ERR_CUDA;
  return cudaDeviceSynchronize() == cudaSuccess ? HBMC_OK : HBMC_ERR_CUDA;
}

hbmc_status hbmc_mlp_train(hbmc_mlp *n, const float *X_dev, const float *T_dev, int32_t B, int32_t steps, float lr,
                           float *loss) {
  if (!n || !X_dev || !T_dev || B < 1 || steps < 0 || !(lr > 0.f)) return HBMC_ERR_INVALID_ARG;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int k = 0; k < steps; ++k) {
    hbmc_status s = mlp_grad(n, X_dev, T_dev, B, n->grad, nullptr);
    if (s != HBMC_OK) return s;
    ++n->step;
    const float c1 = 1.f - powf(b1, (float)n->step), c2 = 1.f - powf(b2, (float)n->step);
    hbmc::k_adam<<<hbmc::nb(n->P, 256), 256>>>(n->p, n->grad, n->m, n->v, n->P, lr, b1, b2, eps, c1, c2);
  }
  hbmc_status s = mlp_grad(n, X_dev, T_dev, B, n->grad, n->loss);
  if (s != HBMC_OK) return s;
  if (loss && cudaMemcpy(loss, n->loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return HBMC_ERR_CUDA;
  return cudaDeviceSynchronize() == cudaSuccess ? HBMC_OK : HBMC_ERR_CUDA;
}

hbmc_status hbmc_features(hbmc_ctx *ctx, float *feat) {
  const hbmc::DeviceLayout *d = nullptr;
  cudaStream_t s;
  int dev;
  bool factored;
  std::string *err;
  if (!feat || !hbmc::ctx_view(ctx, &d, &s, &dev, &factored, &err)) return HBMC_ERR_INVALID_ARG;
  if (d->w != 32 || !d->rec_a) {
    *err = "features: needs a context built with w = 32";
    return HBMC_ERR_INVALID_ARG;
  }
  float *fd = nullptr;
  if (cudaMalloc(&fd, sizeof(float) * hbmc::kFeat) != cudaSuccess) return HBMC_ERR_OOM;
  hbmc_status st = hbmc::features_on_device(*d, 1, nullptr, nullptr, nullptr, fd, s, *err);
  if (st == HBMC_OK && cudaMemcpy(feat, fd, sizeof(float) * hbmc::kFeat, cudaMemcpyDeviceToHost) != cudaSuccess)
    st = HBMC_ERR_CUDA;
  cudaFree(fd);
  return st;
}

hbmc_status hbmc_predict_shift(hbmc_ctx *ctx, hbmc_mlp *net, double *shift, float *predicted) {
  if (!ctx || !net || !shift) return HBMC_ERR_INVALID_ARG;
  if (net->D != hbmc::kFeat + 1) {
    net->err = "predict_shift: the network must take the features plus the shift code";
    return HBMC_ERR_INVALID_ARG;
  }
  const hbmc::DeviceLayout *d = nullptr;
  cudaStream_t s;
  int dev;
  bool factored;
  std::string *err;
  if (!hbmc::ctx_view(ctx, &d, &s, &dev, &factored, &err)) return HBMC_ERR_INVALID_ARG;
  const int ncand = HBMC_SHIFT_GRID;
  float *fd = nullptr, *X = nullptr, *out = nullptr;
  hbmc_status st = HBMC_OK;
  if (cudaMalloc(&fd, sizeof(float) * hbmc::kFeat) != cudaSuccess ||
      cudaMalloc(&X, sizeof(float) * ncand * (hbmc::kFeat + 1)) != cudaSuccess ||
      cudaMalloc(&out, sizeof(float) * ncand) != cudaSuccess)
    st = HBMC_ERR_OOM;
  if (st == HBMC_OK) st = hbmc::features_on_device(*d, 1, nullptr, nullptr, nullptr, fd, s, *err);
  std::vector<float> pred(ncand);
  if (st == HBMC_OK) {
    hbmc::k_candidates<<<1, 32>>>(fd, ncand, X);
    hbmc::k_mlp_forward<<<hbmc::nb(ncand, 4), 128>>>(mlp_view(net), X, ncand, out, nullptr, nullptr);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(pred.data(), out, sizeof(float) * ncand, cudaMemcpyDeviceToHost) != cudaSuccess)
      st = HBMC_ERR_CUDA;
  }
  cudaFree(fd);
  cudaFree(X);
  cudaFree(out);
  if (st != HBMC_OK) return st;
  int best = 0;
  for (int c = 1; c < ncand; ++c)
    if (pred[c] < pred[best]) best = c;  // ties keep the smaller shift
  *shift = grid_shift(best);
  if (predicted)
    for (int c = 0; c < ncand; ++c) predicted[c] = pred[c];
  return HBMC_OK;
}

double hbmc_shift_grid(int32_t c) { return grid_shift(c); }

hbmc_status hbmc_ic0_auto(hbmc_ctx *ctx, hbmc_mlp *net, double *shift_used, int32_t *fallback) {
  if (!ctx || !shift_used) return HBMC_ERR_INVALID_ARG;
  if (fallback) *fallback = 0;
  int first = 0;
  if (net) {
    double a = 0.0;
    hbmc_status st = hbmc_predict_shift(ctx, net, &a, nullptr);
    if (st != HBMC_OK) return st;
    st = hbmc_ic0(ctx, a, nullptr);
    if (st == HBMC_OK) {
      *shift_used = a;
      return HBMC_OK;
    }
    if (st != HBMC_ERR_NOT_SPD_PIVOT) return st;
    if (fallback) *fallback = 1;
    // plain rule from the smallest shift larger than the failed one
    while (first < HBMC_SHIFT_GRID && grid_shift(first) <= a) ++first;
  }
  for (int c = first; c < HBMC_SHIFT_GRID; ++c) {
    const hbmc_status st = hbmc_ic0(ctx, grid_shift(c), nullptr);
    if (st == HBMC_OK) {
      *shift_used = grid_shift(c);
      return HBMC_OK;
    }
    if (st != HBMC_ERR_NOT_SPD_PIVOT) return st;
  }
  return HBMC_ERR_NOT_SPD_PIVOT;
}

}  // extern "C"

// C ABI of libhbmc.so: context lifetime, device layout upload, IC(0), the
// preconditioner and the CG solve (CUDA graph with a device-side while node,
// or a host-driven loop).
#include <cuda_runtime.h>

#include <climits>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hbmc.h"
#include "hbmc_internal.h"
#include "kernels.h"

using hbmc::DeviceLayout;
using hbmc::HostLayout;
using hbmc::Scalars;

namespace hbmc {
hbmc_status finish_device_ctx(hbmc_ctx *ctx);
}

struct hbmc_ctx {
  HostLayout h;
  DeviceLayout d;
  hbmc_options opt{};
  mutable std::string err;  // set by the getters that take a const context too
  int device = 0;
  bool host_only = false;
  bool factored = false;
  int factor_kind = 0;  // 1 IC(0), 2 ILU(0)
  int32_t precision = HBMC_PREC_F64;
  cudaStream_t stream = nullptr;     // user stream (nullptr = legacy default)
  cudaStream_t cap[2] = {nullptr, nullptr};  // private streams used for graph capture
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaGraph_t bgraph[2] = {nullptr, nullptr};  // BiCGStab solve graphs per precision
  cudaGraphExec_t bexec[2] = {nullptr, nullptr};
  Scalars *h_sc = nullptr;           // page-locked mirror of the device scalars
  double *stage_b = nullptr, *stage_x = nullptr;  // device staging for hbmc_iccg_host
  std::vector<void *> allocs;
  int64_t last_iters = 0;
  int64_t last_launches = 0;
};

namespace {

thread_local std::string g_err;

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

hbmc_status set_err(const hbmc_ctx *c, hbmc_status s, const std::string &msg) {
  if (c) c->err = msg; else g_err = msg;
  return s;
}

hbmc_status cuda_err(hbmc_ctx *c, cudaError_t e, const char *what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return set_err(c, e == cudaErrorMemoryAllocation ? HBMC_ERR_OOM : HBMC_ERR_CUDA, m);
}

#define CK(call)                                               \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return cuda_err(ctx, e_, #call);    \
  } while (0)

template <class T>
hbmc_status dalloc(hbmc_ctx *ctx, T *&p, size_t count) {
  p = nullptr;
  size_t bytes = (count ? count : 1) * sizeof(T);
  void *q = nullptr;
  CK(cudaMalloc(&q, bytes));
  ctx->allocs.push_back(q);
  ctx->d.bytes += bytes;
  CK(cudaMemset(q, 0, bytes));
  p = static_cast<T *>(q);
  return HBMC_OK;
}

template <class T>
hbmc_status dupload(hbmc_ctx *ctx, T *&p, const std::vector<T> &v) {
  hbmc_status s = dalloc(ctx, p, v.size());
  if (s != HBMC_OK) return s;
  if (!v.empty()) CK(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return HBMC_OK;
}

#define TRY(expr)                          \
  do {                                     \
    hbmc_status s_ = (expr);               \
    if (s_ != HBMC_OK) return s_;          \
  } while (0)

hbmc_status upload(hbmc_ctx *ctx) {
  const HostLayout &h = ctx->h;
  DeviceLayout &d = ctx->d;
  d.n = h.n;
  d.n_pad = h.n_pad;
  d.nnz_lower = h.nnz_lower;
  d.bs = h.bs;
  d.w = h.w;
  d.nc = h.nc;
  d.tile_ptr = h.tile_ptr;
  std::vector<int32_t> pi32(h.pi.begin(), h.pi.end());
  TRY(dupload(ctx, d.inv, h.inv));
  TRY(dupload(ctx, d.pi, pi32));
  TRY(dupload(ctx, d.a_ptr, h.a_ptr));
  TRY(dupload(ctx, d.a_col, h.a_col));
  TRY(dupload(ctx, d.a_val, h.a_val));
  if (h.split_piece > 0) {
    d.split = 1;
    d.n_virt = (int64_t)(h.sp_ptr.size() - 1) * h.w;
    TRY(dupload(ctx, d.sh_ptr, h.sh_ptr));
    TRY(dupload(ctx, d.sh_col, h.sh_col));
    TRY(dupload(ctx, d.sh_val, h.sh_val));
    TRY(dupload(ctx, d.sp_ptr, h.sp_ptr));
    TRY(dupload(ctx, d.sp_col, h.sp_col));
    TRY(dupload(ctx, d.sp_val, h.sp_val));
    TRY(dupload(ctx, d.sl_mask, h.sl_mask));
    TRY(dupload(ctx, d.sl_first, h.sl_first));
    TRY(dupload(ctx, d.cmb_ptr, h.cmb_ptr));
    TRY(dupload(ctx, d.cmb_slot, h.cmb_slot));
    TRY(dalloc(ctx, d.tsum, (size_t)std::max<int64_t>(d.n_virt, 1)));
  }
  if (h.vslice_cost > 0 && h.split_piece <= 0) {
    d.vslice = 1;
    TRY(dupload(ctx, d.vs_c, h.vs_c));
    TRY(dupload(ctx, d.vs_first, h.vs_first));
    TRY(dupload(ctx, d.vs_ptr, h.vs_ptr));
    TRY(dupload(ctx, d.vs_col, h.vs_col));
    TRY(dupload(ctx, d.vs_val, h.vs_val));
  }
  TRY(dupload(ctx, d.fo_ptr, h.fo_ptr));
  TRY(dupload(ctx, d.fi_ptr, h.fi_ptr));
  TRY(dupload(ctx, d.bo_ptr, h.bo_ptr));
  TRY(dupload(ctx, d.bi_ptr, h.bi_ptr));
  TRY(dupload(ctx, d.fo_col, h.fo_col));
  TRY(dupload(ctx, d.bo_col, h.bo_col));
  TRY(dupload(ctx, d.fi_m, h.fi_m));
  TRY(dupload(ctx, d.bi_m, h.bi_m));
  TRY(dalloc(ctx, d.fo_val, h.fo_col.size()));
  TRY(dalloc(ctx, d.bo_val, h.bo_col.size()));
  TRY(dalloc(ctx, d.fi_val, h.fi_m.size()));
  TRY(dalloc(ctx, d.bi_val, h.bi_m.size()));
  TRY(dalloc(ctx, d.fo_val32, h.fo_col.size()));
  TRY(dalloc(ctx, d.bo_val32, h.bo_col.size()));
  TRY(dalloc(ctx, d.fi_val32, h.fi_m.size()));
  TRY(dalloc(ctx, d.bi_val32, h.bi_m.size()));
  TRY(dalloc(ctx, d.dinv, h.n_pad));
  TRY(dalloc(ctx, d.dinv32, h.n_pad));
  d.dinvb = d.dinv;
  d.dinvb32 = d.dinv32;
  d.nonsym = h.nonsym ? 1 : 0;
  if (h.nonsym) {
    TRY(dalloc(ctx, d.dinvb, h.n_pad));
    TRY(dalloc(ctx, d.dinvb32, h.n_pad));
    TRY(dupload(ctx, d.uaval, h.uaval));
    TRY(dupload(ctx, d.urp, h.urp));
    TRY(dupload(ctx, d.uci, h.uci));
    TRY(dupload(ctx, d.upos, h.upos));
    TRY(dalloc(ctx, d.uval, h.nnz_lower));
    TRY(dalloc(ctx, d.udiag, h.n_pad));
  }
  TRY(dupload(ctx, d.lrp, h.lrp));
  TRY(dupload(ctx, d.lci, h.lci));
  TRY(dupload(ctx, d.laval, h.laval));
  TRY(dupload(ctx, d.adiag, h.adiag));
  TRY(dalloc(ctx, d.lval, h.nnz_lower));
  TRY(dalloc(ctx, d.ldiag, h.n_pad));
  TRY(dupload(ctx, d.lmap_f, h.lmap_f));
  TRY(dupload(ctx, d.lmap_b, h.lmap_b));
  // unpadded runs of the loader-thread sweeps: only layouts that carry them
  // (the batched solver's merged layout does not; its pointers stay null and
  // the scatter and the sweeps then skip them)
  const bool have_x = h.fx_ptr.size() == (size_t)h.ntiles + 1 && h.bx_ptr.size() == (size_t)h.ntiles + 1 &&
                      h.lmapx_f.size() == (size_t)h.nnz_lower && h.lmapx_b.size() == (size_t)h.nnz_lower &&
                      h.nnz_lower > 0;
  if (have_x) {
    TRY(dupload(ctx, d.fx_ptr, h.fx_ptr));
    TRY(dupload(ctx, d.bx_ptr, h.bx_ptr));
    TRY(dupload(ctx, d.fx_rel, h.fx_rel));
    TRY(dupload(ctx, d.bx_rel, h.bx_rel));
    TRY(dupload(ctx, d.fx_col, h.fx_col));
    TRY(dupload(ctx, d.bx_col, h.bx_col));
    TRY(dupload(ctx, d.lmapx_f, h.lmapx_f));
    TRY(dupload(ctx, d.lmapx_b, h.lmapx_b));
    TRY(dalloc(ctx, d.fx_val, h.fx_col.size()));
    TRY(dalloc(ctx, d.bx_val, h.bx_col.size()));
    TRY(dalloc(ctx, d.fx_val32, h.fx_col.size()));
    TRY(dalloc(ctx, d.bx_val32, h.bx_col.size()));
    TRY(dalloc(ctx, d.ucnt, (size_t)std::max<int64_t>(h.ntiles, 1)));
  }
  const size_t nv = (size_t)(h.n_pad + hbmc::kGuard);
  TRY(dalloc(ctx, d.b, nv));
  TRY(dalloc(ctx, d.x, nv));
  TRY(dalloc(ctx, d.r, nv));
  TRY(dalloc(ctx, d.z, nv));
  TRY(dalloc(ctx, d.p, nv));
  TRY(dalloc(ctx, d.q, nv));
  TRY(dalloc(ctx, d.y, nv));
  TRY(dalloc(ctx, d.t, nv));
  TRY(dalloc(ctx, d.y32, nv));
  TRY(dalloc(ctx, d.z32, nv));
  if (h.nonsym) {
    TRY(dalloc(ctx, d.rh, nv));
    TRY(dalloc(ctx, d.sv, nv));
    TRY(dalloc(ctx, d.ph, nv));
  }
  CK(cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, ctx->device));
  while ((1 << d.lw) < d.w) ++d.lw;
  hbmc::sweep_geometry(h, d, ctx->opt.sweep_tpb);
  // 2 named TMA-fed persistent warp-specialized kernels, since retired
  // (bit-identical to the others and never faster); it runs as 0
  d.sweep_kernel = ctx->opt.sweep_kernel == 2 ? 0 : ctx->opt.sweep_kernel;
  d.rec_ints = h.rec_ints;
  if (h.ntiles > 0) {
    TRY(dupload(ctx, d.rec_f, h.rec_f));
    TRY(dupload(ctx, d.rec_b, h.rec_b));
    TRY(dupload(ctx, d.rec_a, h.rec_a));
  }
  hbmc::plan_warp_kernels(h, d);
  CK(hbmc::setup_warp_kernels());
  hbmc::plan_tw_kernels(h, d);
  CK(hbmc::setup_tw_kernels());
  hbmc::plan_spmv_tma(h, d);
  CK(hbmc::setup_spmv_tma());
  hbmc::plan_wide_kernels(h, d);
  CK(hbmc::setup_wide_kernels());
  if (have_x && h.w == 32) {
    hbmc::DagTables t;
    if (hbmc::dag_host_tables(h, t)) {
      TRY(dupload(ctx, d.dag_unit_color, t.ucolor));
      TRY(dupload(ctx, d.dag_color_units, t.color_units));
      TRY(dalloc(ctx, d.dag_color_done, 2 * (size_t)h.nc));
      TRY(dupload(ctx, d.dag_counted, t.counted));
      TRY(dalloc(ctx, d.dag_exit, 2));
      TRY(dupload(ctx, d.dep_ptr_f, t.ptr_f));
      TRY(dupload(ctx, d.dep_f, t.dep_f));
      TRY(dupload(ctx, d.dep_ptr_b, t.ptr_b));
      TRY(dupload(ctx, d.dep_b, t.dep_b));
      TRY(dupload(ctx, d.dag_order_b, t.order_b));
      TRY(dalloc(ctx, d.dag_flag_f, (size_t)h.ntiles));
      TRY(dalloc(ctx, d.dag_flag_b, (size_t)h.ntiles));
      TRY(dalloc(ctx, d.dag_abort, 2));
      TRY(dalloc(ctx, d.dag_ticket, 2));
      hbmc::plan_dag_kernels(h, d);
      CK(hbmc::setup_dag_kernels());
      CK(hbmc::dag_occupancy(d));
    }
  }
  hbmc::plan_sor(h, d);
  CK(hbmc::setup_sor());
  CK(hbmc::setup_persistent());
  if (h.nc > 0) TRY(dupload(ctx, d.tile_ptr_dev, h.tile_ptr));
  TRY(dalloc(ctx, d.pbar, 4));
  d.part_len = hbmc::partials_needed(d);
  TRY(dalloc(ctx, d.part, (size_t)d.part_len));
  TRY(dalloc(ctx, d.hist, (size_t)hbmc::kHistCap));
  TRY(dalloc(ctx, d.sc, 1));
  TRY(dalloc(ctx, ctx->stage_b, (size_t)h.n));
  TRY(dalloc(ctx, ctx->stage_x, (size_t)h.n));
  CK(cudaMallocHost(&ctx->h_sc, sizeof(Scalars)));
  std::memset(ctx->h_sc, 0, sizeof(Scalars));
  CK(cudaStreamCreateWithFlags(&ctx->cap[0], cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&ctx->cap[1], cudaStreamNonBlocking));
  CK(cudaDeviceSynchronize());
  return HBMC_OK;
}

hbmc_status need_device(hbmc_ctx *ctx) {
  if (!ctx) return set_err(nullptr, HBMC_ERR_INVALID_ARG, "null context");
  if (ctx->host_only) return set_err(ctx, HBMC_ERR_NO_DEVICE, "context was built with host_only");
  return HBMC_OK;
}

// Capture the whole solve as one graph: init, a while node running one CG
// iteration per pass (its condition is cleared on the device when the solve
// is done), then the permutation out and the true residual.
hbmc_status build_graph(hbmc_ctx *ctx, int prec, bool bicg) {
  const DeviceLayout &d = ctx->d;
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  (bicg ? ctx->bgraph : ctx->graph)[prec] = g;
  cudaGraphConditionalHandle handle;
  CK(cudaGraphConditionalHandleCreate(&handle, g, 1, cudaGraphCondAssignDefault));
  cudaStream_t s = ctx->cap[0], s2 = ctx->cap[1];
  CK(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  if (bicg) hbmc::enqueue_bcg_init(d, s);
  else hbmc::enqueue_init(d, prec, s);
  cudaStreamCaptureStatus st;
  const cudaGraphNode_t *deps = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, nullptr, &deps, nullptr, &ndeps);
  if (e != cudaSuccess) {
    cudaGraph_t junk;
    cudaStreamEndCapture(s, &junk);
    return cuda_err(ctx, e, "cudaStreamGetCaptureInfo");
  }
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t loop;
  std::vector<cudaGraphNode_t> dv(deps, deps + ndeps);
  e = cudaGraphAddNode(&loop, g, dv.data(), nullptr, dv.size(), &cp);
  if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(s, &loop, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) {
    cudaGraph_t junk;
    cudaStreamEndCapture(s, &junk);
    return cuda_err(ctx, e, "adding the CG while node");
  }
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(s2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t eb = cudaSuccess;
    if (bicg) eb = hbmc::enqueue_bcg_body(d, prec, s2, true, handle);
    else hbmc::enqueue_body(d, prec, s2, true, handle);
    e = cudaStreamEndCapture(s2, &body);
    if (e == cudaSuccess) e = eb;
  }
  if (e != cudaSuccess) {
    cudaGraph_t junk;
    cudaStreamEndCapture(s, &junk);
    return cuda_err(ctx, e, "capturing the CG iteration");
  }
  hbmc::enqueue_final(d, s);
  CK(cudaStreamEndCapture(s, &g));
  CK(cudaGetLastError());
  CK(cudaGraphInstantiate(&(bicg ? ctx->bexec : ctx->exec)[prec], g, 0));
  return HBMC_OK;
}

hbmc_status solve_dev(hbmc_ctx *ctx, const double *b_dev, double *x_dev, double tol, int64_t maxit,
                      int64_t *iters, double *relres, double *true_relres, bool bicg = false) {
  if (iters) *iters = 0;
  if (relres) *relres = 0.0;
  if (true_relres) *true_relres = 0.0;
  if (!(tol > 0.0) || maxit < 0) return set_err(ctx, HBMC_ERR_INVALID_ARG, "tol must be > 0 and maxit >= 0");
  if (ctx->h.n == 0) {
    ctx->last_iters = 0;
    return HBMC_OK;
  }
  if (!b_dev || !x_dev) return set_err(ctx, HBMC_ERR_INVALID_ARG, "null vector");
  if (!ctx->factored) return set_err(ctx, HBMC_ERR_NOT_FACTORED, "no factorization has succeeded on this context");
  if (!bicg && ctx->factor_kind != 1)
    return set_err(ctx, HBMC_ERR_INVALID_ARG, "CG needs the IC(0) factor of a symmetric matrix: use hbmc_bicgstab");
  const int prec = ctx->precision;
  const DeviceLayout &d = ctx->d;
  Scalars init;
  std::memset(&init, 0, sizeof init);
  init.tol = tol;
  init.maxit = maxit;
  init.bad_row = LLONG_MAX;
  init.user_b = b_dev;
  init.user_x = x_dev;
  *ctx->h_sc = init;
  CK(cudaMemcpyAsync(d.sc, ctx->h_sc, sizeof(Scalars), cudaMemcpyHostToDevice, ctx->stream));
  const bool persistent =
      !bicg && ctx->opt.loop_mode == HBMC_LOOP_PERSISTENT && hbmc::persistent_usable(d, prec);
  if (persistent) {
    hbmc::enqueue_gather_in(d, nullptr, d.b, 0, ctx->stream);
    hbmc::enqueue_gather_in(d, nullptr, d.x, 1, ctx->stream);
    CK(hbmc::enqueue_persistent(d, prec, ctx->stream));
    hbmc::enqueue_final(d, ctx->stream);
  } else if (ctx->opt.loop_mode != HBMC_LOOP_HOST) {
    cudaGraphExec_t *ex = bicg ? ctx->bexec : ctx->exec;
    if (!ex[prec]) TRY(build_graph(ctx, prec, bicg));
    CK(cudaGraphLaunch(ex[prec], ctx->stream));
  } else {
    if (bicg) hbmc::enqueue_bcg_init(d, ctx->stream);
    else hbmc::enqueue_init(d, prec, ctx->stream);
    const int every = ctx->opt.check_every > 0 ? ctx->opt.check_every : 16;
    for (int64_t k = 0;; k += every) {
      for (int t = 0; t < every; ++t) {
        if (bicg) CK(hbmc::enqueue_bcg_body(d, prec, ctx->stream, false, 0));
        else hbmc::enqueue_body(d, prec, ctx->stream, false, 0);
      }
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(ctx->h_sc, d.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      if (ctx->h_sc->done) break;
    }
    hbmc::enqueue_final(d, ctx->stream);
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(ctx->h_sc, d.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const Scalars &r = *ctx->h_sc;
  ctx->last_iters = r.iters;
  {
    // init: 2 gathers, residual, n_c + n_c sweeps, p = z; per CG iteration:
    // SpMV, x/r update, 2 n_c sweeps, p update; after: gather, residual.
    // In graph mode the body runs `iters` times (at least once); in host
    // mode it is enqueued in groups of check_every.
    // BiCGStab: init = 2 gathers, residual, start; per iteration 7 kernels
    // and two preconditioner applications (4 n_c sweeps).
    // Row-split SpMV: one more launch for the pieces; the fused last color
    // of the preconditioner: one launch fewer.
    const int64_t sw = hbmc::sweep_launches(d, prec), pc = hbmc::precond_launches(d, prec);
    const int64_t per = bicg ? 7 + 4 * sw : 3 + pc + (d.split && d.n_virt > 0 ? 1 : 0);
    int64_t passes = r.iters > 0 ? r.iters : 1;
    if (ctx->opt.loop_mode == HBMC_LOOP_HOST) {
      const int64_t every = ctx->opt.check_every > 0 ? ctx->opt.check_every : 16;
      passes = (passes + every - 1) / every * every;
    }
    ctx->last_launches = persistent ? 5 : (bicg ? 4 : 4 + pc) + passes * per + 2;
  }
  if (iters) *iters = r.iters;
  if (relres) *relres = r.relres;
  if (true_relres) *true_relres = r.true_relres;
  if (r.timeout) return set_err(ctx, HBMC_ERR_TIMEOUT, "a bounded device-side wait ran out");
  switch (r.status) {
    case hbmc::ST_CONVERGED: return HBMC_OK;
    case hbmc::ST_MAXIT: return set_err(ctx, HBMC_NOT_CONVERGED, "maxit reached before the tolerance");
    case hbmc::ST_BREAKDOWN: return set_err(ctx, HBMC_ERR_BREAKDOWN, "CG breakdown: p.q or r.z not positive and finite");
    default: return set_err(ctx, HBMC_ERR_CUDA, "solve ended without a final status");
  }
}

}  // namespace

extern "C" {

void hbmc_default_options(hbmc_options *opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof *opt);
  opt->blocking = HBMC_BLOCK_ALGEBRAIC;
  opt->precision = HBMC_PREC_F64;
  opt->loop_mode = HBMC_LOOP_GRAPH;
  opt->device = -1;
  opt->check_every = 16;
}

const char *hbmc_status_string(hbmc_status s) {
  switch (s) {
    case HBMC_OK: return "HBMC_OK";
    case HBMC_ERR_INVALID_ARG: return "HBMC_ERR_INVALID_ARG";
    case HBMC_ERR_NOT_SPD_PIVOT: return "HBMC_ERR_NOT_SPD_PIVOT";
    case HBMC_ERR_BREAKDOWN: return "HBMC_ERR_BREAKDOWN";
    case HBMC_NOT_CONVERGED: return "HBMC_NOT_CONVERGED";
    case HBMC_ERR_TIMEOUT: return "HBMC_ERR_TIMEOUT";
    case HBMC_ERR_CUDA: return "HBMC_ERR_CUDA";
    case HBMC_ERR_OOM: return "HBMC_ERR_OOM";
    case HBMC_ERR_NOT_FACTORED: return "HBMC_ERR_NOT_FACTORED";
    case HBMC_ERR_NO_DEVICE: return "HBMC_ERR_NO_DEVICE";
  }
  return "HBMC_UNKNOWN_STATUS";
}

const char *hbmc_last_error(const hbmc_ctx *ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

hbmc_status hbmc_build(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                       int32_t bs, int32_t w, const hbmc_options *opt, hbmc_ctx **out) {
  if (!out) return set_err(nullptr, HBMC_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  g_err.clear();
  hbmc_options o;
  hbmc_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != HBMC_PREC_F64 && o.precision != HBMC_PREC_F32)
    return set_err(nullptr, HBMC_ERR_INVALID_ARG, "unknown precision");
  if (o.loop_mode != HBMC_LOOP_GRAPH && o.loop_mode != HBMC_LOOP_HOST && o.loop_mode != HBMC_LOOP_PERSISTENT)
    return set_err(nullptr, HBMC_ERR_INVALID_ARG, "unknown loop mode");
  if (o.sell_split < 0 || o.sell_split_cost < 0)
    return set_err(nullptr, HBMC_ERR_INVALID_ARG, "sell_split and sell_split_cost must be >= 0");
  if (o.sell_split > 0 && w > 32)
    return set_err(nullptr, HBMC_ERR_INVALID_ARG, "row splitting needs w <= 32");
  if (o.sell_vslice < 0) return set_err(nullptr, HBMC_ERR_INVALID_ARG, "sell_vslice must be >= 0");
  if (o.sweep_kernel < 0 || o.sweep_kernel > 8)
    return set_err(nullptr, HBMC_ERR_INVALID_ARG, "sweep_kernel must be in 0..8");
  if (o.sweep_tpb < 0 || (o.sweep_tpb & (o.sweep_tpb - 1)) || (int64_t)o.sweep_tpb * w > 256)
    return set_err(nullptr, HBMC_ERR_INVALID_ARG, "sweep_tpb must be 0 or a power of two with sweep_tpb * w <= 256");
  hbmc_ctx *ctx = nullptr;
  try {
    ctx = new hbmc_ctx();
  } catch (...) {
    return set_err(nullptr, HBMC_ERR_OOM, "host allocation failed");
  }
  ctx->opt = o;
  ctx->host_only = o.host_only != 0;
  ctx->precision = o.precision;
  hbmc_status s;
  try {
    s = hbmc::build_host(n, row_ptr, col, val, bs, w, o, ctx->h, ctx->err);
  } catch (const std::bad_alloc &) {
    s = HBMC_ERR_OOM;
    ctx->err = "host allocation failed";
  }
  if (s != HBMC_OK) {
    g_err = ctx->err;
    delete ctx;
    return s;
  }
  if (!ctx->host_only) {
    s = hbmc::finish_device_ctx(ctx);
    if (s != HBMC_OK) {
      g_err = ctx->err;
      hbmc_destroy(ctx);
      return s;
    }
  }
  *out = ctx;
  return HBMC_OK;
}

void hbmc_destroy(hbmc_ctx *ctx) {
  if (!ctx) return;
  if (!ctx->host_only) {
    DeviceGuard guard(ctx->device);
    cudaDeviceSynchronize();
    for (int k = 0; k < 2; ++k) {
      if (ctx->exec[k]) cudaGraphExecDestroy(ctx->exec[k]);
      if (ctx->graph[k]) cudaGraphDestroy(ctx->graph[k]);
      if (ctx->bexec[k]) cudaGraphExecDestroy(ctx->bexec[k]);
      if (ctx->bgraph[k]) cudaGraphDestroy(ctx->bgraph[k]);
      if (ctx->cap[k]) cudaStreamDestroy(ctx->cap[k]);
    }
    for (void *p : ctx->allocs) cudaFree(p);
    if (ctx->h_sc) cudaFreeHost(ctx->h_sc);
  }
  delete ctx;
}

hbmc_status hbmc_debug_convert(const double *d_in, float *f_out, const float *f_in, double *d_out, int64_t n,
                               void *stream) {
  if (n < 0 || (n > 0 && (!d_in || !f_out || !f_in || !d_out))) return HBMC_ERR_INVALID_ARG;
  if (n == 0) return HBMC_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  hbmc::enqueue_convert_ieee(d_in, f_out, f_in, d_out, n, s);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return HBMC_ERR_CUDA;
  return HBMC_OK;
}

hbmc_status hbmc_debug_stall(hbmc_ctx *ctx, int64_t unit, double wait_s) {
  TRY(need_device(ctx));
  if (unit >= ctx->h.ntiles) return set_err(ctx, HBMC_ERR_INVALID_ARG, "unit beyond the last level-1 block");
  if (!(wait_s <= 1e6)) return set_err(ctx, HBMC_ERR_INVALID_ARG, "wait_s must be a number of seconds <= 1e6");
  DeviceGuard guard(ctx->device);
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->d.dag_stall = unit < 0 ? -1 : unit;
  ctx->d.dag_wait_ns = wait_s > 0.0 ? (uint64_t)(wait_s * 1e9) : 4000000000ull;
  // the kernels' arguments are fixed inside a captured graph
  for (int k = 0; k < 2; ++k) {
    if (ctx->exec[k]) cudaGraphExecDestroy(ctx->exec[k]);
    if (ctx->graph[k]) cudaGraphDestroy(ctx->graph[k]);
    if (ctx->bexec[k]) cudaGraphExecDestroy(ctx->bexec[k]);
    if (ctx->bgraph[k]) cudaGraphDestroy(ctx->bgraph[k]);
    ctx->exec[k] = nullptr;
    ctx->graph[k] = nullptr;
    ctx->bexec[k] = nullptr;
    ctx->bgraph[k] = nullptr;
  }
  return HBMC_OK;
}

hbmc_status hbmc_info(const hbmc_ctx *ctx, hbmc_info_t *info) {
  if (!ctx || !info) return set_err(nullptr, HBMC_ERR_INVALID_ARG, "null argument");
  const HostLayout &h = ctx->h;
  std::memset(info, 0, sizeof *info);
  info->n = h.n;
  info->n_pad = h.n_pad;
  info->nnz = h.nnz;
  info->nnz_lower = h.n ? (h.nnz - h.n) / 2 : 0;
  info->bs = h.bs;
  info->w = h.w;
  info->nc = h.nc;
  info->nblocks = h.nblocks;
  info->ntiles = h.ntiles;
  info->sell_entries_a = (int64_t)h.a_col.size();
  info->sell_entries_l = (int64_t)(h.fo_col.size() + h.fi_m.size());
  info->sell_entries_u = (int64_t)(h.bo_col.size() + h.bi_m.size());
  info->precision = ctx->precision;
  info->factored = ctx->factored ? 1 : 0;
  info->device_bytes = ctx->d.bytes;
  info->last_iters = ctx->last_iters;
  info->last_launches = ctx->last_launches;
  info->split_rows = h.split_rows;
  info->split_pieces = h.split_pieces;
  info->sell_entries_split = h.split_piece > 0 ? (int64_t)(h.sh_col.size() + h.sp_col.size()) : 0;
  info->sell_entries_vslice = h.vslice_cost > 0 ? (int64_t)h.vs_col.size() : 0;
  return HBMC_OK;
}

hbmc_status hbmc_get_split(const hbmc_ctx *ctx, int32_t *head) {
  if (!ctx) return set_err(nullptr, HBMC_ERR_INVALID_ARG, "null context");
  const HostLayout &h = ctx->h;
  if (h.split_piece <= 0) return set_err(ctx, HBMC_ERR_INVALID_ARG, "the context was built without row splitting");
  if (head && !h.split_head.empty()) std::memcpy(head, h.split_head.data(), sizeof(int32_t) * h.split_head.size());
  return HBMC_OK;
}

hbmc_status hbmc_get_vslice(const hbmc_ctx *ctx, int32_t *height) {
  if (!ctx) return set_err(nullptr, HBMC_ERR_INVALID_ARG, "null context");
  const HostLayout &h = ctx->h;
  if (h.vslice_cost <= 0) return set_err(ctx, HBMC_ERR_INVALID_ARG, "the context was built without sell_vslice");
  if (height)
    for (size_t s = 0; s < h.vs_c.size(); ++s) height[s] = h.vs_c[s];
  return HBMC_OK;
}

hbmc_status hbmc_get_dag_deps(const hbmc_ctx *ctx, int32_t dir, int64_t *ptr, int32_t *dep, int64_t cap,
                              int64_t *count) {
  if (!ctx) return set_err(nullptr, HBMC_ERR_INVALID_ARG, "null context");
  if (dir != 0 && dir != 1) return set_err(ctx, HBMC_ERR_INVALID_ARG, "dir must be 0 (forward) or 1 (backward)");
  hbmc::DagTables t;
  try {
    if (!hbmc::dag_host_tables(ctx->h, t))
      return set_err(ctx, HBMC_ERR_INVALID_ARG,
                     "the dependency-driven sweeps need w = 32 and at least one level-1 block");
  } catch (const std::bad_alloc &) {
    return set_err(ctx, HBMC_ERR_OOM, "host allocation failed");
  }
  const std::vector<int64_t> &p = dir == 0 ? t.ptr_f : t.ptr_b;
  const std::vector<int32_t> &v = dir == 0 ? t.dep_f : t.dep_b;
  if (count) *count = (int64_t)v.size();
  if (dep && cap < (int64_t)v.size())
    return set_err(ctx, HBMC_ERR_INVALID_ARG, "cap is smaller than the number of entries");
  if (ptr) std::memcpy(ptr, p.data(), sizeof(int64_t) * p.size());
  if (dep && !v.empty()) std::memcpy(dep, v.data(), sizeof(int32_t) * v.size());
  return HBMC_OK;
}

hbmc_status hbmc_get_ordering(const hbmc_ctx *ctx, int64_t *pi, int64_t *color_ptr, int64_t *block_of,
                              int32_t *block_color) {
  if (!ctx) return set_err(nullptr, HBMC_ERR_INVALID_ARG, "null context");
  const HostLayout &h = ctx->h;
  if (pi && h.n) std::memcpy(pi, h.pi.data(), sizeof(int64_t) * h.n);
  if (color_ptr) std::memcpy(color_ptr, h.color_ptr.data(), sizeof(int64_t) * (h.nc + 1));
  if (block_of && h.n) std::memcpy(block_of, h.block_of.data(), sizeof(int64_t) * h.n);
  if (block_color && h.nblocks) std::memcpy(block_color, h.block_color.data(), sizeof(int32_t) * h.nblocks);
  return HBMC_OK;
}

hbmc_status hbmc_get_matrix(const hbmc_ctx *ctx, int64_t *row_ptr, int32_t *col, double *val) {
  if (!ctx) return set_err(nullptr, HBMC_ERR_INVALID_ARG, "null context");
  const HostLayout &h = ctx->h;
  if (row_ptr) std::memcpy(row_ptr, h.rp.data(), sizeof(int64_t) * h.rp.size());
  if (col && !h.ci.empty()) std::memcpy(col, h.ci.data(), sizeof(int32_t) * h.ci.size());
  if (val && !h.av.empty()) std::memcpy(val, h.av.data(), sizeof(double) * h.av.size());
  return HBMC_OK;
}

hbmc_status hbmc_set_stream(hbmc_ctx *ctx, void *stream) {
  if (!ctx) return set_err(nullptr, HBMC_ERR_INVALID_ARG, "null context");
  ctx->stream = static_cast<cudaStream_t>(stream);
  return HBMC_OK;
}

hbmc_status hbmc_set_precision(hbmc_ctx *ctx, int32_t precision) {
  if (!ctx) return set_err(nullptr, HBMC_ERR_INVALID_ARG, "null context");
  if (precision != HBMC_PREC_F64 && precision != HBMC_PREC_F32)
    return set_err(ctx, HBMC_ERR_INVALID_ARG, "unknown precision");
  ctx->precision = precision;
  return HBMC_OK;
}

hbmc_status hbmc_ic0(hbmc_ctx *ctx, double shift, int64_t *bad_row) {
  if (bad_row) *bad_row = -1;
  TRY(need_device(ctx));
  if (!(shift > -1.0) || !(shift < 1e300)) return set_err(ctx, HBMC_ERR_INVALID_ARG, "shift must be > -1 and finite");
  if (ctx->h.nonsym)
    return set_err(ctx, HBMC_ERR_INVALID_ARG, "the context was built for nonsymmetric values: use hbmc_ilu0");
  ctx->factored = false;
  ctx->factor_kind = 0;
  if (ctx->h.n == 0) {
    ctx->factored = true;
    ctx->factor_kind = 1;
    return HBMC_OK;
  }
  DeviceGuard guard(ctx->device);
  hbmc::enqueue_ic0(ctx->d, shift, ctx->stream);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(ctx->h_sc, ctx->d.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const long long bad = ctx->h_sc->bad_row;
  if (bad != LLONG_MAX) {
    int64_t orig = (bad >= 0 && bad < ctx->h.n_pad) ? ctx->h.inv[bad] : -1;
    if (bad_row) *bad_row = orig;
    char buf[128];
    std::snprintf(buf, sizeof buf, "IC(0) pivot not positive at row %lld (reordered %lld)",
                  (long long)orig, (long long)bad);
    return set_err(ctx, HBMC_ERR_NOT_SPD_PIVOT, buf);
  }
  hbmc::enqueue_scatter_factor(ctx->d, true, ctx->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->factored = true;
  ctx->factor_kind = 1;
  return HBMC_OK;
}

hbmc_status hbmc_ilu0(hbmc_ctx *ctx, double shift, int64_t *bad_row) {
  if (bad_row) *bad_row = -1;
  TRY(need_device(ctx));
  if (!(shift > -1.0) || !(shift < 1e300)) return set_err(ctx, HBMC_ERR_INVALID_ARG, "shift must be > -1 and finite");
  if (!ctx->h.nonsym)
    return set_err(ctx, HBMC_ERR_INVALID_ARG, "hbmc_ilu0 needs a context built with opt.nonsymmetric = 1");
  ctx->factored = false;
  ctx->factor_kind = 0;
  if (ctx->h.n == 0) {
    ctx->factored = true;
    ctx->factor_kind = 2;
    return HBMC_OK;
  }
  DeviceGuard guard(ctx->device);
  const DeviceLayout &d = ctx->d;
  hbmc::enqueue_ilu0(d, shift, ctx->stream);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(ctx->h_sc, d.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const long long bad = ctx->h_sc->bad_row;
  if (bad != LLONG_MAX) {
    int64_t orig = (bad >= 0 && bad < ctx->h.n_pad) ? ctx->h.inv[bad] : -1;
    if (bad_row) *bad_row = orig;
    char buf[128];
    std::snprintf(buf, sizeof buf, "ILU(0) pivot zero or not finite at row %lld (reordered %lld)",
                  (long long)orig, (long long)bad);
    return set_err(ctx, HBMC_ERR_NOT_SPD_PIVOT, buf);
  }
  hbmc::enqueue_unit_dinv(d, ctx->stream);
  hbmc::enqueue_scatter_factor(d, true, ctx->stream, d.uval);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->factored = true;
  ctx->factor_kind = 2;
  return HBMC_OK;
}

hbmc_status hbmc_get_factor_u(const hbmc_ctx *ctx_c, double *upper) {
  hbmc_ctx *ctx = const_cast<hbmc_ctx *>(ctx_c);
  TRY(need_device(ctx));
  if (!ctx->factored || ctx->factor_kind != 2) return set_err(ctx, HBMC_ERR_NOT_FACTORED, "no ILU(0) factor");
  if (!upper) return set_err(ctx, HBMC_ERR_INVALID_ARG, "null output");
  DeviceGuard guard(ctx->device);
  const HostLayout &h = ctx->h;
  CK(cudaStreamSynchronize(ctx->stream));
  std::vector<double> uv(h.nnz_lower);
  if (h.nnz_lower) CK(cudaMemcpy(uv.data(), ctx->d.uval, sizeof(double) * h.nnz_lower, cudaMemcpyDeviceToHost));
  std::memset(upper, 0, sizeof(double) * h.ci.size());
  for (int64_t e = 0; e < h.nnz_lower; ++e) upper[h.u_to_abar[e]] = uv[e];
  return HBMC_OK;
}

hbmc_status hbmc_get_factor(const hbmc_ctx *ctx_c, double *lower, double *diag) {
  hbmc_ctx *ctx = const_cast<hbmc_ctx *>(ctx_c);
  TRY(need_device(ctx));
  if (!ctx->factored) return set_err(ctx, HBMC_ERR_NOT_FACTORED, "no factor");
  DeviceGuard guard(ctx->device);
  const HostLayout &h = ctx->h;
  CK(cudaStreamSynchronize(ctx->stream));
  if (lower) {
    std::vector<double> lv(h.nnz_lower);
    if (h.nnz_lower) CK(cudaMemcpy(lv.data(), ctx->d.lval, sizeof(double) * h.nnz_lower, cudaMemcpyDeviceToHost));
    std::memset(lower, 0, sizeof(double) * h.ci.size());
    for (int64_t e = 0; e < h.nnz_lower; ++e) lower[h.l_to_abar[e]] = lv[e];
  }
  if (diag && h.n_pad)
    CK(cudaMemcpy(diag, ctx->factor_kind == 2 ? ctx->d.udiag : ctx->d.ldiag, sizeof(double) * h.n_pad,
                  cudaMemcpyDeviceToHost));
  return HBMC_OK;
}

hbmc_status hbmc_precond(hbmc_ctx *ctx, const double *r_dev, double *z_dev) {
  TRY(need_device(ctx));
  if (!ctx->factored) return set_err(ctx, HBMC_ERR_NOT_FACTORED, "hbmc_ic0 has not succeeded on this context");
  if (ctx->h.n == 0) return HBMC_OK;
  if (!r_dev || !z_dev) return set_err(ctx, HBMC_ERR_INVALID_ARG, "null vector");
  DeviceGuard guard(ctx->device);
  const DeviceLayout &d = ctx->d;
  hbmc::enqueue_gather_in(d, r_dev, d.r, -1, ctx->stream);
  hbmc::enqueue_precond(d, ctx->precision, d.r, 0, false, ctx->stream);
  hbmc::enqueue_gather_out(d, d.z, z_dev, false, ctx->stream);
  CK(cudaGetLastError());
  return HBMC_OK;
}

hbmc_status hbmc_iccg(hbmc_ctx *ctx, const double *b_dev, double *x_dev, double tol, int64_t maxit,
                      int64_t *iters, double *relres, double *true_relres) {
  TRY(need_device(ctx));
  DeviceGuard guard(ctx->device);
  return solve_dev(ctx, b_dev, x_dev, tol, maxit, iters, relres, true_relres);
}

hbmc_status hbmc_bicgstab(hbmc_ctx *ctx, const double *b_dev, double *x_dev, double tol, int64_t maxit,
                          int64_t *iters, double *relres, double *true_relres) {
  TRY(need_device(ctx));
  if (ctx->h.n && !ctx->h.nonsym)
    return set_err(ctx, HBMC_ERR_INVALID_ARG, "hbmc_bicgstab needs a context built with opt.nonsymmetric = 1");
  DeviceGuard guard(ctx->device);
  return solve_dev(ctx, b_dev, x_dev, tol, maxit, iters, relres, true_relres, true);
}

hbmc_status hbmc_iccg_host(hbmc_ctx *ctx, const double *b_host, double *x_host, double tol,
                           int64_t maxit, int64_t *iters, double *relres, double *true_relres) {
  TRY(need_device(ctx));
  if (ctx->h.n && (!b_host || !x_host)) return set_err(ctx, HBMC_ERR_INVALID_ARG, "null vector");
  DeviceGuard guard(ctx->device);
  const size_t bytes = sizeof(double) * (size_t)ctx->h.n;
  if (bytes) {
    CK(cudaMemcpyAsync(ctx->stage_b, b_host, bytes, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->stage_x, x_host, bytes, cudaMemcpyHostToDevice, ctx->stream));
  }
  hbmc_status s = solve_dev(ctx, ctx->stage_b, ctx->stage_x, tol, maxit, iters, relres, true_relres);
  if (bytes && (s == HBMC_OK || s == HBMC_NOT_CONVERGED || s == HBMC_ERR_BREAKDOWN)) {
    CK(cudaMemcpyAsync(x_host, ctx->stage_x, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return s;
}

hbmc_status hbmc_residual_history(const hbmc_ctx *ctx_c, double *hist, int64_t cap, int64_t *count) {
  hbmc_ctx *ctx = const_cast<hbmc_ctx *>(ctx_c);
  if (count) *count = 0;
  TRY(need_device(ctx));
  if (!hist || cap < 0) return set_err(ctx, HBMC_ERR_INVALID_ARG, "bad history buffer");
  if (ctx->h.n == 0) return HBMC_OK;
  int64_t m = ctx->last_iters + 1;
  if (m > hbmc::kHistCap) m = hbmc::kHistCap;
  if (m > cap) m = cap;
  DeviceGuard guard(ctx->device);
  CK(cudaStreamSynchronize(ctx->stream));
  if (m > 0) CK(cudaMemcpy(hist, ctx->d.hist, sizeof(double) * m, cudaMemcpyDeviceToHost));
  if (count) *count = m;
  return HBMC_OK;
}

hbmc_status hbmc_fwd_bar(hbmc_ctx *ctx, const double *r_dev, double *y_dev) {
  TRY(need_device(ctx));
  if (!ctx->factored) return set_err(ctx, HBMC_ERR_NOT_FACTORED, "no factor");
  if (ctx->h.n == 0) return HBMC_OK;
  if (!r_dev || !y_dev) return set_err(ctx, HBMC_ERR_INVALID_ARG, "null vector");
  DeviceGuard guard(ctx->device);
  const DeviceLayout &d = ctx->d;
  const size_t bytes = sizeof(double) * (size_t)d.n_pad;
  CK(cudaMemcpyAsync(d.r, r_dev, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  hbmc::enqueue_fwd(d, ctx->precision, d.r, false, ctx->stream);
  if (ctx->precision == HBMC_PREC_F64)
    CK(cudaMemcpyAsync(y_dev, d.y, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  else
    hbmc::enqueue_widen(d.y32, y_dev, d.n_pad, ctx->stream);
  CK(cudaGetLastError());
  return HBMC_OK;
}

hbmc_status hbmc_bwd_bar(hbmc_ctx *ctx, const double *y_dev, double *z_dev) {
  TRY(need_device(ctx));
  if (!ctx->factored) return set_err(ctx, HBMC_ERR_NOT_FACTORED, "no factor");
  if (ctx->h.n == 0) return HBMC_OK;
  if (!y_dev || !z_dev) return set_err(ctx, HBMC_ERR_INVALID_ARG, "null vector");
  DeviceGuard guard(ctx->device);
  const DeviceLayout &d = ctx->d;
  const size_t bytes = sizeof(double) * (size_t)d.n_pad;
  if (ctx->precision == HBMC_PREC_F64)
    CK(cudaMemcpyAsync(d.y, y_dev, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  else
    hbmc::enqueue_narrow(y_dev, d.y32, d.n_pad, ctx->stream);
  hbmc::enqueue_bwd(d, ctx->precision, d.r, 0, false, ctx->stream);
  CK(cudaMemcpyAsync(z_dev, d.z, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaGetLastError());
  return HBMC_OK;
}

hbmc_status hbmc_spmv_bar(hbmc_ctx *ctx, const double *p_dev, double *q_dev) {
  TRY(need_device(ctx));
  if (ctx->h.n == 0) return HBMC_OK;
  if (!p_dev || !q_dev) return set_err(ctx, HBMC_ERR_INVALID_ARG, "null vector");
  DeviceGuard guard(ctx->device);
  const DeviceLayout &d = ctx->d;
  const size_t bytes = sizeof(double) * (size_t)d.n_pad;
  CK(cudaMemcpyAsync(d.t, p_dev, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  hbmc::enqueue_spmv(d, d.t, d.q, false, ctx->stream);
  CK(cudaMemcpyAsync(q_dev, d.q, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaGetLastError());
  return HBMC_OK;
}

hbmc_status hbmc_sor_bar(hbmc_ctx *ctx, const double *b_dev, double *x_dev, double omega, int32_t sweeps,
                         int32_t symmetric) {
  TRY(need_device(ctx));
  if (!(omega > 0.0 && omega < 2.0) || sweeps < 0)
    return set_err(ctx, HBMC_ERR_INVALID_ARG, "omega must be in (0, 2) and sweeps >= 0");
  if (ctx->h.n == 0 || sweeps == 0) return HBMC_OK;
  if (!b_dev || !x_dev) return set_err(ctx, HBMC_ERR_INVALID_ARG, "null vector");
  DeviceGuard guard(ctx->device);
  const DeviceLayout &d = ctx->d;
  if (!hbmc::sor_usable(d)) return set_err(ctx, HBMC_ERR_INVALID_ARG, "a level-1 block's rows do not fit in shared memory");
  const size_t bytes = sizeof(double) * (size_t)d.n_pad;
  CK(cudaMemcpyAsync(d.b, b_dev, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaMemcpyAsync(d.x, x_dev, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  hbmc::enqueue_sor(d, d.x, d.b, omega, sweeps, symmetric != 0, ctx->stream);
  CK(cudaMemcpyAsync(x_dev, d.x, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaGetLastError());
  return HBMC_OK;
}

hbmc_status hbmc_sor(hbmc_ctx *ctx, const double *b_dev, double *x_dev, double omega, int32_t sweeps,
                     int32_t symmetric, double *relres) {
  if (relres) *relres = 0.0;
  TRY(need_device(ctx));
  if (!(omega > 0.0 && omega < 2.0) || sweeps < 0)
    return set_err(ctx, HBMC_ERR_INVALID_ARG, "omega must be in (0, 2) and sweeps >= 0");
  if (ctx->h.n == 0) return HBMC_OK;
  if (!b_dev || !x_dev) return set_err(ctx, HBMC_ERR_INVALID_ARG, "null vector");
  DeviceGuard guard(ctx->device);
  const DeviceLayout &d = ctx->d;
  if (!hbmc::sor_usable(d)) return set_err(ctx, HBMC_ERR_INVALID_ARG, "a level-1 block's rows do not fit in shared memory");
  Scalars init;
  std::memset(&init, 0, sizeof init);
  init.tol = 0.0;
  init.bad_row = LLONG_MAX;
  *ctx->h_sc = init;
  CK(cudaMemcpyAsync(d.sc, ctx->h_sc, sizeof(Scalars), cudaMemcpyHostToDevice, ctx->stream));
  hbmc::enqueue_gather_in(d, b_dev, d.b, 2, ctx->stream);
  hbmc::enqueue_gather_in(d, x_dev, d.x, 2, ctx->stream);
  hbmc::enqueue_sor(d, d.x, d.b, omega, sweeps, symmetric != 0, ctx->stream);
  hbmc::enqueue_gather_out(d, d.x, x_dev, false, ctx->stream);
  hbmc::enqueue_relres(d, ctx->stream);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(ctx->h_sc, d.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (relres) *relres = ctx->h_sc->relres;
  return HBMC_OK;
}

hbmc_status hbmc_profile_kernels(hbmc_ctx *ctx, int32_t reps, double *ms) {
  TRY(need_device(ctx));
  if (!ms || reps < 1) return set_err(ctx, HBMC_ERR_INVALID_ARG, "bad arguments");
  for (int k = 0; k < 5; ++k) ms[k] = 0.0;
  if (!ctx->factored) return set_err(ctx, HBMC_ERR_NOT_FACTORED, "no factor");
  if (ctx->h.n == 0) return HBMC_OK;
  DeviceGuard guard(ctx->device);
  const DeviceLayout &d = ctx->d;
  cudaStream_t s = ctx->stream;
  const int prec = ctx->precision;
  // A scalar block that keeps every kernel running: not done, alpha = beta =
  // 0 (the vector updates leave x, r, p unchanged), rho = 1, a large maxit.
  Scalars sc;
  std::memset(&sc, 0, sizeof sc);
  sc.rho = 1.0;
  sc.bnorm = 1.0;
  sc.tol = 0.0;
  sc.maxit = 1ll << 60;
  sc.bad_row = LLONG_MAX;
  *ctx->h_sc = sc;
  CK(cudaMemcpyAsync(d.sc, ctx->h_sc, sizeof(Scalars), cudaMemcpyHostToDevice, s));
  cudaEvent_t ev[2];
  CK(cudaEventCreate(&ev[0]));
  CK(cudaEventCreate(&ev[1]));
  for (int k = 0; k < 5; ++k) {
    auto run = [&]() {
      switch (k) {
        case 0: hbmc::enqueue_fwd(d, prec, d.r, true, s); break;
        case 1: hbmc::enqueue_bwd(d, prec, d.r, 2, true, s); break;
        case 2: hbmc::enqueue_spmv(d, d.p, d.q, true, s); break;
        case 3: hbmc::enqueue_update_xr(d, s); break;
        case 4: hbmc::enqueue_update_p(d, s); break;
      }
    };
    for (int w = 0; w < 2; ++w) run();
    CK(cudaEventRecord(ev[0], s));
    for (int r = 0; r < reps; ++r) run();
    CK(cudaEventRecord(ev[1], s));
    CK(cudaEventSynchronize(ev[1]));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, ev[0], ev[1]));
    ms[k] = (double)t / reps;
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  CK(cudaMemcpyAsync(ctx->h_sc, d.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (ctx->h_sc->done) return set_err(ctx, HBMC_ERR_BREAKDOWN, "profiling run hit a breakdown; timings invalid");
  return HBMC_OK;
}

}  // extern "C"

namespace hbmc {

// Device half of context creation: pick the device, set kernel attributes
// and upload the host layout.
hbmc_status finish_device_ctx(hbmc_ctx *ctx) {
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
    return set_err(ctx, HBMC_ERR_NO_DEVICE, "no CUDA device");
  int dev = ctx->opt.device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  if (dev >= ndev) return set_err(ctx, HBMC_ERR_INVALID_ARG, "device ordinal out of range");
  ctx->device = dev;
  DeviceGuard guard(dev);
  cudaError_t e = hbmc::setup_kernels();
  if (e != cudaSuccess) return cuda_err(ctx, e, "setup_kernels");
  return upload(ctx);
}

// A device context around a host layout built elsewhere (the batched solver).
hbmc_status make_ctx_from_layout(HostLayout &&h, const hbmc_options &opt, hbmc_ctx **out, std::string &err) {
  *out = nullptr;
  hbmc_ctx *ctx = nullptr;
  try {
    ctx = new hbmc_ctx();
  } catch (...) {
    err = "host allocation failed";
    return HBMC_ERR_OOM;
  }
  ctx->opt = opt;
  ctx->host_only = false;
  ctx->precision = opt.precision;
  ctx->h = std::move(h);
  hbmc_status s = finish_device_ctx(ctx);
  if (s != HBMC_OK) {
    err = ctx->err;
    hbmc_destroy(ctx);
    return s;
  }
  *out = ctx;
  return HBMC_OK;
}

// Read-only view of a context for entry points defined in other translation
// units; returns false for a null or host-only context.
bool ctx_view(hbmc_ctx *ctx, const DeviceLayout **d, cudaStream_t *stream, int *device,
              bool *factored, std::string **err) {
  if (!ctx || ctx->host_only) return false;
  *d = &ctx->d;
  *stream = ctx->stream;
  *device = ctx->device;
  *factored = ctx->factored;
  *err = &ctx->err;
  return true;
}

}  // namespace hbmc

// Enqueue sequences of the HBMC-ICCG kernels (defined in kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "hbmc_internal.h"

namespace hbmc {

cudaError_t setup_kernels();
int64_t partials_needed(const DeviceLayout &d);

void enqueue_gather_in(const DeviceLayout &d, const double *src, double *dst, int which, cudaStream_t s);
void enqueue_gather_out(const DeviceLayout &d, const double *src, double *dst, bool to_user, cudaStream_t s);
void enqueue_widen(const float *src, double *dst, int64_t n, cudaStream_t s);
void enqueue_narrow(const double *src, float *dst, int64_t n, cudaStream_t s);
void enqueue_spmv(const DeviceLayout &d, const double *p, double *q, bool dot, cudaStream_t s);
void enqueue_fwd(const DeviceLayout &d, int prec, const double *r, bool check_done, cudaStream_t s);
void enqueue_bwd(const DeviceLayout &d, int prec, const double *r, int dot_mode, bool check_done, cudaStream_t s);
void enqueue_init(const DeviceLayout &d, int prec, cudaStream_t s);
void enqueue_body(const DeviceLayout &d, int prec, cudaStream_t s, bool use_cond, cudaGraphConditionalHandle h);
void enqueue_final(const DeviceLayout &d, cudaStream_t s);
void enqueue_ic0(const DeviceLayout &d, double shift, cudaStream_t s);
void enqueue_scatter_factor(const DeviceLayout &d, bool f32, cudaStream_t s);

}  // namespace hbmc

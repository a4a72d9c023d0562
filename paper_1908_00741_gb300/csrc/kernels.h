// Enqueue sequences of the HBMC-ICCG kernels (defined in kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "hbmc_internal.h"

namespace hbmc {

cudaError_t setup_kernels();
void sweep_geometry(const HostLayout &h, DeviceLayout &d, int tpb);
int64_t partials_needed(const DeviceLayout &d);

// Warp-per-unit kernels (sweep_warp.cu)
void plan_warp_kernels(const HostLayout &h, DeviceLayout &d);
cudaError_t setup_warp_kernels();
bool warp_usable(const DeviceLayout &d, bool fwd, int prec);
bool warp_spmv_usable(const DeviceLayout &d);
int64_t warp_partials_needed(const DeviceLayout &d);
void enqueue_fwd_warp(const DeviceLayout &d, int prec, const double *r, bool check_done, cudaStream_t s);
void enqueue_bwd_warp(const DeviceLayout &d, int prec, const double *r, int dot_mode, bool check_done,
                      cudaStream_t s);
void enqueue_spmv_warp(const DeviceLayout &d, const double *p, double *q, bool dot, cudaStream_t s);

// Warp-per-unit substitution kernels with bulk-copy staging, bs 4 or 8 (sweep_tw.cu)
void plan_tw_kernels(const HostLayout &h, DeviceLayout &d);
cudaError_t setup_tw_kernels();
bool tw_usable(const DeviceLayout &d, bool fwd, int prec);
int64_t tw_partials_needed(const DeviceLayout &d);
unsigned tw_color_grid(const DeviceLayout &d, int c);
bool fb_tw_usable(const DeviceLayout &d, int prec);
void launch_fb_tw_last(const DeviceLayout &d, int prec, const double *r, int dot_mode, bool check_done,
                       int64_t part_off, bool last, int64_t part_total, cudaStream_t s);
void enqueue_precond(const DeviceLayout &d, int prec, const double *r, int dot_mode, bool check_done,
                     cudaStream_t s);
void launch_fwd_tw_color(const DeviceLayout &d, int prec, int c, const double *r, bool check_done, cudaStream_t s);
void launch_bwd_tw_color(const DeviceLayout &d, int prec, int c, const double *r, int dot_mode, bool check_done,
                         int64_t part_off, bool last, int64_t part_total, cudaStream_t s);

// One CUDA block per level-1 block with loader threads (sweep_wide.cu): for
// colors with few level-1 blocks, where one warp per block leaves the GPU idle
void plan_wide_kernels(const HostLayout &h, DeviceLayout &d);
cudaError_t setup_wide_kernels();
bool wide_usable(const DeviceLayout &d, bool fwd, int prec);
bool wide_all(const DeviceLayout &d);
bool wide_preferred(const DeviceLayout &d, bool fwd, int c);
unsigned wide_color_grid(const DeviceLayout &d, int c);
void launch_fwd_wide_color(const DeviceLayout &d, int prec, int c, const double *r, bool check_done, cudaStream_t s);
void launch_bwd_wide_color(const DeviceLayout &d, int prec, int c, const double *r, int dot_mode, bool check_done,
                           int64_t part_off, bool last, int64_t part_total, cudaStream_t s);

// Dependency-driven sweeps: every color in one launch (sweep_dag.cu).
// Host tables: per level-1 block what it waits for (forward / backward), the
// backward sweep's order, level-1 block -> color, color -> level-1 blocks.
struct DagTables {
  std::vector<int64_t> ptr_f, ptr_b, color_units;
  std::vector<int32_t> dep_f, dep_b, order_b, ucolor;
  std::vector<uint8_t> counted;  // per color, forward then backward: some level-1 block waits on its counter
};
bool dag_host_tables(const HostLayout &h, DagTables &t);
void plan_dag_kernels(const HostLayout &h, DeviceLayout &d);
cudaError_t setup_dag_kernels();
cudaError_t dag_occupancy(DeviceLayout &d);
bool dag_usable(const DeviceLayout &d, bool fwd, int prec);
bool dag_selected(const DeviceLayout &d, int prec);
void enqueue_fwd_dag(const DeviceLayout &d, int prec, const double *r, bool check_done, cudaStream_t s);
void enqueue_bwd_dag(const DeviceLayout &d, int prec, const double *r, int dot_mode, bool check_done,
                     cudaStream_t s);

// launches of one forward (or backward) sweep, and of one preconditioner application
int64_t sweep_launches(const DeviceLayout &d, int prec);
int64_t precond_launches(const DeviceLayout &d, int prec);

// Bulk-copy-fed SpMV, w = 32 (spmv_tma.cu)
void plan_spmv_tma(const HostLayout &h, DeviceLayout &d);
cudaError_t setup_spmv_tma();
bool spmv_tma_usable(const DeviceLayout &d);
int64_t spmv_tma_partials_needed(const DeviceLayout &d);
void enqueue_spmv_tma(const DeviceLayout &d, const double *p, double *q, bool dot, cudaStream_t s);

// The whole CG solve as one persistent cooperative kernel (persistent.cu)
cudaError_t setup_persistent();
bool persistent_usable(const DeviceLayout &d, int prec);
cudaError_t enqueue_persistent(const DeviceLayout &d, int prec, cudaStream_t s);

// SOR / symmetric SOR sweeps on the HBMC ordering (sor.cu)
void plan_sor(const HostLayout &h, DeviceLayout &d);
cudaError_t setup_sor();
bool sor_usable(const DeviceLayout &d);
void enqueue_sor(const DeviceLayout &d, double *x, const double *b, double omega, int64_t sweeps, bool symmetric,
                 cudaStream_t s);

void enqueue_gather_in(const DeviceLayout &d, const double *src, double *dst, int which, cudaStream_t s);
void enqueue_gather_out(const DeviceLayout &d, const double *src, double *dst, bool to_user, cudaStream_t s);
void enqueue_widen(const float *src, double *dst, int64_t n, cudaStream_t s);
void enqueue_narrow(const double *src, float *dst, int64_t n, cudaStream_t s);
void enqueue_convert_ieee(const double *din, float *fout, const float *fin, double *dout, int64_t n,
                          cudaStream_t s);
// q = A p (with p.q and alpha when dot): the row-split layout when the
// context has one, else enqueue_spmv_plain.
void enqueue_spmv(const DeviceLayout &d, const double *p, double *q, bool dot, cudaStream_t s);
// q = A p on the unsplit SELL layout.
void enqueue_spmv_plain(const DeviceLayout &d, const double *p, double *q, bool dot, cudaStream_t s);
void enqueue_fwd(const DeviceLayout &d, int prec, const double *r, bool check_done, cudaStream_t s);
void enqueue_bwd(const DeviceLayout &d, int prec, const double *r, int dot_mode, bool check_done, cudaStream_t s);
void enqueue_init(const DeviceLayout &d, int prec, cudaStream_t s);
void enqueue_body(const DeviceLayout &d, int prec, cudaStream_t s, bool use_cond, cudaGraphConditionalHandle h);
void enqueue_final(const DeviceLayout &d, cudaStream_t s);
void enqueue_relres(const DeviceLayout &d, cudaStream_t s);
void enqueue_update_xr(const DeviceLayout &d, cudaStream_t s);
void enqueue_update_p(const DeviceLayout &d, cudaStream_t s);
void enqueue_ic0(const DeviceLayout &d, double shift, cudaStream_t s);
void enqueue_scatter_factor(const DeviceLayout &d, bool f32, cudaStream_t s, const double *bval = nullptr);
void enqueue_reset_bad_row(const DeviceLayout &d, cudaStream_t s);

// ILU(0) and BiCGStab for nonsymmetric values (bicgstab.cu)
void enqueue_ilu0(const DeviceLayout &d, double shift, cudaStream_t s);
void enqueue_unit_dinv(const DeviceLayout &d, cudaStream_t s);
void enqueue_bcg_init(const DeviceLayout &d, cudaStream_t s);
cudaError_t enqueue_bcg_body(const DeviceLayout &d, int prec, cudaStream_t s, bool use_cond,
                             cudaGraphConditionalHandle h);
int64_t bcg_partials_needed(const DeviceLayout &d);

}  // namespace hbmc

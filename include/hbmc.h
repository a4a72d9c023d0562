/*
 * hbmc.h - C ABI of the GB300 HBMC-ICCG solver (libhbmc.so).
 *
 * Solves A x = b for a sparse symmetric positive definite A by IC(0)-
 * preconditioned CG whose forward and backward substitutions run under
 * hierarchical block multi-color (HBMC) ordering (Iwashita, Li, Fukaya,
 * arXiv:1908.00741).  Problem statement: Section 2, Eq. "org"; IC(0)-CG with
 * A symmetric positive (semi-)definite.
 *
 * Conventions for every entry point
 *   - Input matrices are host CSR: row_ptr int64[n+1] (row_ptr[0] = 0),
 *     col int32[nnz] strictly ascending inside each row, val double[nnz];
 *     both triangles stored, numerically symmetric (a_ij == a_ji exactly),
 *     positive diagonal present in every row.  The library copies them;
 *     the caller keeps ownership.
 *   - Vectors passed as *_dev are caller-owned CUDA device pointers of
 *     doubles on the context's device.  "Original ordering" vectors have
 *     length n; "reordered" vectors (the *_bar step functions) have length
 *     n_pad in HBMC order.
 *   - All GPU work is enqueued on the context's stream (hbmc_set_stream;
 *     default: the legacy default stream).  Functions that return numeric
 *     results synchronize that stream before returning; hbmc_precond and the
 *     step functions are asynchronous.
 *   - Errors are reported only through the returned status; no exception,
 *     abort or device trap crosses the ABI.  hbmc_last_error() gives a
 *     one-line description of the most recent failure on a context.
 *   - A context is not thread safe; use one context per host thread.
 */
#ifndef HBMC_H_
#define HBMC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hbmc_status {
  HBMC_OK = 0,
  HBMC_ERR_INVALID_ARG = 1,   /* bad sizes, pointers, CSR or options */
  HBMC_ERR_NOT_SPD_PIVOT = 2, /* IC(0) met a pivot that is not positive and finite */
  HBMC_ERR_BREAKDOWN = 3,     /* CG: p.q or r.z not positive and finite */
  HBMC_NOT_CONVERGED = 4,     /* maxit reached before the tolerance */
  HBMC_ERR_TIMEOUT = 5,       /* a bounded device-side wait ran out */
  HBMC_ERR_CUDA = 6,          /* a CUDA runtime call failed */
  HBMC_ERR_OOM = 7,           /* device or host allocation failed */
  HBMC_ERR_NOT_FACTORED = 8,  /* solve requested before a successful hbmc_ic0 */
  HBMC_ERR_NO_DEVICE = 9      /* context built with host_only, or no CUDA device */
} hbmc_status;

/* Blocking rule for the BMC blocks (Section 4.1). */
enum {
  HBMC_BLOCK_ALGEBRAIC = 0, /* Section 5.1: seed = minimal-numbered unassigned unknown,
                               grown by the minimal-numbered unassigned neighbour */
  HBMC_BLOCK_BOXES = 1      /* geometric bx*by*bz boxes of a lexicographic grid (x fastest) */
};

/* Arithmetic of the preconditioner substitutions.  The CG recurrences, dot
 * products, SpMV and the IC(0) factorization are always FP64. */
enum { HBMC_PREC_F64 = 0, HBMC_PREC_F32 = 1 };

/* How the CG loop is driven on the device. */
enum {
  HBMC_LOOP_GRAPH = 0, /* one CUDA graph launch per solve; a device-side while node
                          runs the iterations, convergence decided on the GPU */
  HBMC_LOOP_HOST = 1,  /* host launches iterations and polls a device flag */
  HBMC_LOOP_PERSISTENT = 2 /* the whole CG solve in one persistent cooperative kernel with
                              grid-wide barriers between the phases: for small systems, whose
                              iterations the launches dominate (w = 32 and no row
                              splitting, else as
                              HBMC_LOOP_GRAPH; BiCGStab runs as HBMC_LOOP_GRAPH) */
};

typedef struct hbmc_options {
  int32_t blocking;  /* HBMC_BLOCK_ALGEBRAIC (default) or HBMC_BLOCK_BOXES */
  int64_t grid[3];   /* nx, ny, nz for HBMC_BLOCK_BOXES (n must equal nx*ny*nz) */
  int32_t box[3];    /* bx, by, bz for HBMC_BLOCK_BOXES (bx*by*bz must equal bs) */
  int32_t precision; /* HBMC_PREC_F64 (default) or HBMC_PREC_F32 */
  int32_t loop_mode; /* HBMC_LOOP_GRAPH (default), HBMC_LOOP_HOST or HBMC_LOOP_PERSISTENT */
  int32_t host_only; /* nonzero: compute the ordering and layouts on the host only,
                        touch no GPU (inspection and CPU tests) */
  int32_t device;    /* CUDA device ordinal; -1 = the current device */
  int32_t check_every; /* HBMC_LOOP_HOST: iterations between flag polls (default 16) */
  int32_t sweep_tpb;   /* level-1 blocks per CUDA block in the substitution kernels;
                          0 = automatic, else a power of two with sweep_tpb * w <= 256 */
  int32_t sweep_kernel; /* substitution kernels: 0 = automatic (8 when the matrix has 8 or
                           more colors and two of its CUDA blocks fit on an SM; else one warp
                           per level-1 block when w = 32 and its runs fit in shared memory --
                           right-hand side, dinv and same-block runs staged by bulk copy when
                           bs is 4 or 8 -- else 1);
                           1 = one CUDA block per level-1 block(s);
                           2 = retired (TMA-fed persistent warp-specialized kernels, removed:
                               bit-identical to the others and never faster); runs as 0;
                           3 = one warp per level-1 block reading its runs with plain loads,
                               and SpMV one warp per level-1 block too (w = 32);
                           4 = one CUDA block of loader threads per level-1 block for every
                               color (automatic under 0, when bs is 4 or 8 and w = 32, for
                               colors whose level-1 blocks average 2048 or more other-color
                               couplings or that have fewer than two level-1 blocks per SM;
                               runs staged by bulk copy when w = 32 and that costs no extra
                               wave of CUDA blocks);
                           5 = the bulk-copy-staged warp kernels of 0 for every color;
                           6 = as 4 with the runs read by plain loads instead of bulk
                               copies (the form 4 uses when w < 32);
                           7 = as 6 with each level-1 block's other-color sums spread over
                               bs CUDA blocks, one per step, the last of which to finish
                               runs the chains (automatic under 0 for colors with fewer
                               than two level-1 blocks per SM whose other-color runs
                               average 12288 or more entries);
                           8 = dependency-driven: each sweep is one launch over every
                               color, one CUDA block per level-1 block; a level-1 block
                               waits only for the level-1 blocks of other colors whose
                               rows it reads (Section 4.3.3's n_c - 1 synchronizations
                               per sweep become per-block flags), needs w = 32 and its
                               runs in shared memory, else as 0.
                           SpMV (w = 32) is fed by bulk copies when a chunk of its slices fits
                           in shared memory, else one thread per row; with 3 it runs one warp
                           per level-1 block. */
  int32_t nonsymmetric; /* 0: A must be symmetric (IC(0), CG); 1: only the pattern must be
                           symmetric and the diagonal nonzero (ILU(0), BiCGStab) */
  int32_t sell_split;   /* row splitting of the CG's SpMV (Section 5.2.2: SELL pads every row
                           of a slice to the slice's longest row; the remedy splits the long
                           rows).  0 = off (default).  P > 0: every slice of w rows gets a head
                           width t in [1, longest row] minimising
                             w*t + sum over rows longer than t of
                                   (length - t) + sell_split_cost * ceil((length - t) / P)
                           (the largest t among equal costs); a row keeps its first t entries
                           in the slice and the rest is cut into pieces of P entries (the last
                           shorter), stored as rows of their own sorted by length.  Each part
                           is summed from zero in ascending column order with fused
                           multiply-adds and the parts' sums are added in order, so the
                           product differs from the unsplit one in rounding only.  Used by
                           the SpMV of hbmc_iccg and hbmc_spmv_bar; the residuals and every
                           other kernel keep the unsplit layout.  Needs w = 32 or less. */
  int32_t sell_split_cost; /* the per-piece cost of the plan above, in entries (0 = 2) */
  int32_t sell_vslice;  /* variable slice height of the CG's SpMV layout (Section 5.2.2 and the
                           conclusions: the other remedy for SELL's padding).  0 = off
                           (default).  K > 0: every slice of w rows is cut into w / C
                           sub-slices of C consecutive rows, C in {w, w/2, w/4}, each padded
                           only to its own longest row; the slice takes the C minimising
                             sum over its sub-slices of C * (longest row) + K * (w / C)
                           (the largest C among equal costs).  Rows keep their order and
                           every row's terms are summed as in the plain SpMV, so the product
                           is bit-identical to it.  Used by the SpMV of hbmc_iccg and
                           hbmc_spmv_bar unless sell_split is set too (row splitting wins). */
} hbmc_options;

/* Fills *opt with the defaults. */
void hbmc_default_options(hbmc_options *opt);

typedef struct hbmc_ctx hbmc_ctx; /* opaque; owns every buffer it allocates */

typedef struct hbmc_info_t {
  int64_t n;          /* unknowns */
  int64_t n_pad;      /* unknowns plus dummies (Section 4.2.1) */
  int64_t nnz;        /* nonzeros of A */
  int64_t nnz_lower;  /* strict lower nonzeros of A = nonzeros of L off the diagonal */
  int32_t bs, w;      /* block size b_s and level-1 width w */
  int32_t nc;         /* colors n_c */
  int64_t nblocks;    /* BMC blocks (before padding) */
  int64_t ntiles;     /* level-1 blocks of all colors (after padding) */
  int64_t sell_entries_a;   /* stored SpMV entries including slice padding */
  int64_t sell_entries_l;   /* stored forward-sweep entries including padding */
  int64_t sell_entries_u;   /* stored backward-sweep entries including padding */
  int32_t precision;
  int32_t factored;   /* 1 after a successful hbmc_ic0 */
  size_t device_bytes;      /* device memory held by the context */
  int64_t last_iters;       /* iterations of the last hbmc_iccg call */
  int64_t last_launches;    /* kernels launched by the last hbmc_iccg call */
  int64_t split_rows;       /* rows cut by the SpMV row splitting (0 without it) */
  int64_t split_pieces;     /* pieces those rows were cut into */
  int64_t sell_entries_split; /* stored entries of the split SpMV layout: heads plus the
                                 pieces' slices, each with its padding (0 without it) */
  int64_t sell_entries_vslice; /* stored entries of the variable-slice-height SpMV layout,
                                  padding included (0 without it) */
} hbmc_info_t;

/*
 * hbmc_build - block, color and reorder A, then lay it out on the device.
 *
 * Section 4.1 (BMC: blocks of bs unknowns, greedy block coloring; the
 * blocking heuristic and greedy coloring of Section 5.1), Section 4.2
 * (level-1 blocks of w consecutive same-color BMC blocks, Eq. "simd-block";
 * secondary reordering; dummy unknowns so every color is a multiple of bs*w),
 * Section 4.3.2 (SELL storage with slice size w).
 *
 * n, row_ptr, col, val: host CSR of A (see conventions).  n == 0 gives a
 * valid empty context.  bs in [1, 64]; w in {1, 2, 4, 8, 16, 32}.
 * opt may be NULL (defaults).  On success *out receives a new context that
 * the caller frees with hbmc_destroy; on failure *out is NULL.
 * Errors: INVALID_ARG (CSR not sorted, not symmetric, missing or
 * non-positive diagonal, bad bs/w/options), OOM, CUDA, NO_DEVICE.
 */
hbmc_status hbmc_build(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                       int32_t bs, int32_t w, const hbmc_options *opt, hbmc_ctx **out);

/* Releases every resource of ctx (NULL is ignored). */
void hbmc_destroy(hbmc_ctx *ctx);

/* One-line description of the last error on ctx (or of the last failed
 * hbmc_build in this thread when ctx is NULL).  Valid until the next call. */
const char *hbmc_last_error(const hbmc_ctx *ctx);

/* Static name of a status code. */
const char *hbmc_status_string(hbmc_status s);

/* Fills *info (the fields of hbmc_info_t above) from ctx; works for host_only
 * contexts.  INVALID_ARG when ctx or info is NULL. */
hbmc_status hbmc_info(const hbmc_ctx *ctx, hbmc_info_t *info);

/*
 * hbmc_get_ordering - copy the host-side ordering out (works for host_only
 * contexts).  pi: int64[n], the position of original unknown i in the padded
 * HBMC numbering (the reordering function pi of Section 3).  color_ptr:
 * int64[nc+1], color c occupies [color_ptr[c], color_ptr[c+1]).  block_of:
 * int64[n] BMC block of each unknown; block_color: int32[nblocks].  Any
 * output pointer may be NULL.
 */
hbmc_status hbmc_get_ordering(const hbmc_ctx *ctx, int64_t *pi, int64_t *color_ptr,
                              int64_t *block_of, int32_t *block_color);

/*
 * hbmc_get_matrix - host copy of Abar = P A P^T (Section 3, Eq. "AB") on the
 * padded index space (dummy rows are identity rows): row_ptr int64[n_pad+1],
 * col int32[nnz + n_pad - n], val double[nnz + n_pad - n], sorted columns.
 */
hbmc_status hbmc_get_matrix(const hbmc_ctx *ctx, int64_t *row_ptr, int32_t *col, double *val);

/*
 * hbmc_get_split - the head width t of every slice of w rows of the split
 * SpMV layout (hbmc_options.sell_split; Section 5.2.2's row splitting):
 * head int32[n_pad / w].  Works for host_only contexts.  INVALID_ARG when the
 * context was built without row splitting.
 */
hbmc_status hbmc_get_split(const hbmc_ctx *ctx, int32_t *head);

/*
 * hbmc_get_vslice - the sub-slice height C of every slice of w rows of the
 * variable-slice-height SpMV layout (hbmc_options.sell_vslice; Section
 * 5.2.2): height int32[n_pad / w].  Works for host_only contexts.
 * INVALID_ARG when the context was built without it.
 */
hbmc_status hbmc_get_vslice(const hbmc_ctx *ctx, int32_t *height);

/*
 * hbmc_get_dag_deps - what each level-1 block of a dependency-driven sweep
 * (sweep_kernel 8, chosen automatically for 8 or more colors) waits for.
 * Section 4.3.3 counts n_c - 1 barriers per substitution; these sweeps
 * replace them by waits on only the level-1 blocks whose rows a level-1
 * block reads through its other-color couplings (Eq. "for3").
 *
 * dir: 0 forward sweep (entries of earlier colors), 1 backward sweep (later
 * colors).  ptr: int64[ntiles + 1], level-1 block u's entries are
 * dep[ptr[u] .. ptr[u + 1]).  An entry v >= 0 is a level-1 block (index into
 * the level-1 blocks of all colors, colors in order); an entry -(c + 1) is
 * color c, whose completion counter replaces the level-1 blocks of that
 * color where u reads more than 16 of them.  Entries are sorted by the first
 * row they cover (forward) or by the row after their last, descending
 * (backward), the order in which the sweep gathers their terms.  dep:
 * int32[cap], may be NULL to query *count (the total number of entries)
 * first; ptr and count may be NULL too.  Works for host_only contexts.
 * INVALID_ARG when w != 32, the context has no level-1 block, dir is not 0
 * or 1, or dep is given with cap < *count (*count is still set).
 */
hbmc_status hbmc_get_dag_deps(const hbmc_ctx *ctx, int32_t dir, int64_t *ptr, int32_t *dep, int64_t cap,
                              int64_t *count);

/* Bind the context to a CUDA stream (a cudaStream_t, e.g. from
 * torch.cuda.current_stream().cuda_stream); NULL = legacy default stream. */
hbmc_status hbmc_set_stream(hbmc_ctx *ctx, void *stream);

/* Switch the substitution arithmetic (HBMC_PREC_F64 or HBMC_PREC_F32).  The
 * FP32 factor is a rounded copy of the FP64 factor made by hbmc_ic0. */
hbmc_status hbmc_set_precision(hbmc_ctx *ctx, int32_t precision);

/*
 * hbmc_ic0 - shifted IC(0) factorization of Abar on the GPU.
 *
 * Section 2, Eq. "ILU" (A ~= L U with L, U on the patterns of the lower and
 * upper triangles of A; for IC(0) U = L^T), with the diagonal shift of the
 * shifted ICCG of Section 5.1: the factored matrix has diagonal
 * (1 + shift) * a_ii and unchanged off-diagonals.  Runs color by color with
 * the same level-1 / lane structure as the substitutions.  shift > -1.
 * bad_row (may be NULL) receives -1 on success, or on HBMC_ERR_NOT_SPD_PIVOT
 * the original index of the first row (in HBMC order) whose pivot was not
 * positive and finite.  Synchronizes the stream.
 */
hbmc_status hbmc_ic0(hbmc_ctx *ctx, double shift, int64_t *bad_row);

/*
 * hbmc_get_factor - host copy of the FP64 factor: lower holds l_ij at the
 * position of each entry of Abar (hbmc_get_matrix layout; 0 for diagonal and
 * upper entries), diag holds l_ii (n_pad).  Either pointer may be NULL.
 */
hbmc_status hbmc_get_factor(const hbmc_ctx *ctx, double *lower, double *diag);

/*
 * hbmc_precond - z = (L L^T)^{-1} r in the original ordering: permute in,
 * forward substitution y = L^{-1} r (Eq. "for") over colors 1..n_c,
 * backward substitution z = L^{-T} y (Eq. "back") over colors n_c..1,
 * permute out.  Color n_c's forward and backward passes may run as one
 * launch (the last color gathers nothing in the backward sweep); the bits
 * are those of the two separate sweeps.  r_dev, z_dev: device double[n] (may not alias).
 * Asynchronous.  Errors: NOT_FACTORED, INVALID_ARG, CUDA.
 */
hbmc_status hbmc_precond(hbmc_ctx *ctx, const double *r_dev, double *z_dev);

/*
 * hbmc_iccg - solve A x = b by IC(0)-preconditioned CG (Section 2; stopping
 * rule of Section 5.1: 2-norm relative residual ||r_k|| / ||b|| < tol, with
 * the recurrence residual).
 *
 * b_dev: device double[n], original ordering.  x_dev: device double[n]; on
 * entry the initial guess, on exit the solution.  tol > 0; maxit >= 0.
 * iters: CG iterations performed (x updates); relres: final recurrence
 * relative residual; true_relres: ||b - A x|| / ||b|| recomputed in FP64
 * after the loop.  Any output pointer may be NULL.  Synchronizes the stream.
 * Returns OK, NOT_CONVERGED (maxit reached; x holds the last iterate),
 * BREAKDOWN, NOT_FACTORED, INVALID_ARG or CUDA.
 */
hbmc_status hbmc_iccg(hbmc_ctx *ctx, const double *b_dev, double *x_dev, double tol, int64_t maxit,
                      int64_t *iters, double *relres, double *true_relres);

/*
 * hbmc_iccg_host - hbmc_iccg with HOST vectors b_host[n] and x_host[n]
 * (x_host is the initial guess on entry).  Copies b and x0 to the device,
 * solves and copies x back, all on the context's stream.  Page-locked host
 * memory gives the fastest copies.
 */
hbmc_status hbmc_iccg_host(hbmc_ctx *ctx, const double *b_host, double *x_host, double tol,
                           int64_t maxit, int64_t *iters, double *relres, double *true_relres);

/*
 * hbmc_residual_history - copy the recurrence relative residuals of the last
 * hbmc_iccg call: hist[0] for the initial guess, hist[k] after iteration k,
 * for k = 0..min(iters, cap-1).  Returns the number written in *count.
 * Recording costs one store per iteration and is always on (up to the
 * capacity fixed at build time, 100000 entries).
 */
hbmc_status hbmc_residual_history(const hbmc_ctx *ctx, double *hist, int64_t cap, int64_t *count);

/*
 * Step functions on reordered, padded vectors (length n_pad, HBMC order),
 * for testing and for callers that keep their vectors in HBMC order.
 * They run the kernels of the solve one at a time and are asynchronous.
 *
 * hbmc_fwd_bar: y = L^{-1} r (Eq. "for"; colors 1..n_c, Eqs. "for2",
 *   "for3"; inside a level-1 block the bs steps of Eqs. "y2-2", "y2-3").
 * hbmc_bwd_bar: z = L^{-T} y (Eq. "back"; colors n_c..1).
 * hbmc_spmv_bar: q = Abar p.
 * In HBMC_PREC_F32 mode the substitutions compute in FP32 and the results
 * are widened to double on output.
 */
hbmc_status hbmc_fwd_bar(hbmc_ctx *ctx, const double *r_dev, double *y_dev);
hbmc_status hbmc_bwd_bar(hbmc_ctx *ctx, const double *y_dev, double *z_dev);
hbmc_status hbmc_spmv_bar(hbmc_ctx *ctx, const double *p_dev, double *q_dev);

/*
 * hbmc_profile_kernels - average device time (ms, CUDA events on the
 * context's stream) of each phase of one CG iteration, each run `reps`
 * times back to back on the context's own vectors: ms[0] forward
 * substitution (all colors), ms[1] backward substitution with the fused r.z
 * (all colors), ms[2] SpMV with the fused p.q, ms[3] x/r update with ||r||,
 * ms[4] p update.  The two sweeps are timed as separate launch sequences;
 * inside a solve the last color's two passes may share one launch (so a
 * solve's preconditioner can take less than ms[0] + ms[1]).  Call it after
 * a solve (the vectors then hold data of the right scale); it leaves the
 * context ready for the next solve.
 * Synchronizes the stream.
 */
hbmc_status hbmc_profile_kernels(hbmc_ctx *ctx, int32_t reps, double *ms);

/*
 * hbmc_debug_stall - test hook for the bounded waits of the
 * dependency-driven sweeps (sweep_kernel 8); the paper has no counterpart.
 * unit >= 0: level-1 block `unit` (0-based, HBMC order) computes its rows
 * but never publishes its completion flag, so every level-1 block that
 * gathers from it waits until wait_s seconds have passed, gives up, and the
 * solve returns HBMC_ERR_TIMEOUT with the context still usable.  unit = -1
 * restores normal operation; wait_s <= 0 restores the default bound (4 s).
 * Takes effect at the next launch; a solve graph captured earlier keeps the
 * values it was captured with, so the hook discards the context's graphs.
 */
hbmc_status hbmc_debug_stall(hbmc_ctx *ctx, int64_t unit, double wait_s);

/*
 * hbmc_debug_convert - test hook for the conversions the FP32 substitutions
 * make between binary64 and binary32 with integer operations (the paper
 * has no counterpart; they keep the conversions off this GPU's FP64 pipe):
 * f_out[i] = d_in[i] rounded to float (to nearest, ties to even) and
 * d_out[i] = f_in[i] widened to double, for i < n.  All four pointers are
 * device arrays of n elements; stream is a cudaStream_t (NULL = legacy
 * default stream).  Synchronizes the stream.  HBMC_ERR_INVALID_ARG for
 * n < 0 or a NULL pointer with n > 0, HBMC_ERR_CUDA on a launch error.
 */
hbmc_status hbmc_debug_convert(const double *d_in, float *f_out, const float *f_in, double *d_out, int64_t n,
                               void *stream);

/*
 * hbmc_ilu0 - ILU(0) of Abar for a context built with opt.nonsymmetric = 1
 * (Section 2: ILU(0) preconditioning; the HBMC ordering makes its
 * substitutions parallel exactly as for IC(0), with U in place of L^T).
 * Abar ~= L U, L unit lower triangular on the pattern of Abar's strict lower
 * triangle, U upper triangular on the pattern of its upper triangle; the
 * diagonal is scaled by (1 + shift).  Row by row in index order, entries in
 * ascending column: w = abar_ij - sum_{k<min(i,j)} l_ik u_kj (one fma per
 * term, k ascending), l_ij = w / u_jj for j < i, u_ij = w for j >= i.
 * Computed color by color on the device (lane = BMC block, as hbmc_ic0).
 * bad_row (may be NULL) gets -1 or the original index of the first row whose
 * pivot u_ii is zero or not finite (status HBMC_ERR_NOT_SPD_PIVOT).
 * hbmc_ic0 is refused on such a context, hbmc_ilu0 on a symmetric one.
 * Synchronizes.
 */
hbmc_status hbmc_ilu0(hbmc_ctx *ctx, double shift, int64_t *bad_row);

/* U of the ILU(0) factor on the positions of Abar's strict upper triangle
 * (host double[nnz of Abar], as hbmc_get_matrix's values; zero elsewhere).
 * hbmc_get_factor returns L and, for an ILU(0) context, the pivots u_ii. */
hbmc_status hbmc_get_factor_u(const hbmc_ctx *ctx, double *upper);

/*
 * hbmc_bicgstab - ILU(0)-preconditioned BiCGStab (right preconditioning,
 * van der Vorst) on Abar for a context built with opt.nonsymmetric = 1 and
 * factored by hbmc_ilu0.  Per iteration: beta = (rho / rho_old)(alpha /
 * omega), p = r + beta (p - omega v), ph = M^{-1} p, v = A ph, alpha = rho /
 * (rh, v), s = r - alpha v (if ||s|| / ||b|| < tol: x += alpha ph and stop),
 * sh = M^{-1} s, t = A sh, omega = (t, s) / (t, t), x += alpha ph + omega sh,
 * r = s - omega t, stop when ||r|| / ||b|| < tol, rho_old = rho, rho = (rh,
 * r); rh = r0.  Vectors, outputs and statuses as hbmc_iccg (HBMC_ERR_BREAKDOWN
 * when rho, (rh, v), (t, t) or omega is zero or not finite).  Honours
 * hbmc_set_precision (FP32 substitutions) and opt.loop_mode.  Synchronizes.
 */
hbmc_status hbmc_bicgstab(hbmc_ctx *ctx, const double *b_dev, double *x_dev, double tol, int64_t maxit,
                          int64_t *iters, double *relres, double *true_relres);

/*
 * hbmc_sor - SOR sweeps on the HBMC ordering (Section 2: the GS and SOR
 * iteration steps are substitutions like IC(0)'s; Section 3.1, Eq. "xj":
 * the equivalent reordering gives the same iterates, so each color's
 * level-1 blocks run in parallel).  Row by row in the reordered order
 * (forward sweep ascending; with symmetric != 0 every sweep is followed by a
 * backward sweep, descending: symmetric SOR):
 *   s = sum_{j != i} abar_ij x_j (ascending column, one fused multiply-add
 *   per term from zero), t = (b_i - s) * (1 / abar_ii),
 *   x_i = fma(omega, t - x_i, x_i).
 * omega = 1 is Gauss-Seidel.  b_dev, x_dev: device doubles of length n in the
 * original ordering; x_dev holds the initial guess on entry and the result
 * on exit.  omega in (0, 2), sweeps >= 0.  relres (host, may be NULL)
 * receives ||b - A x|| / ||b|| after the sweeps (0 for b = 0).  Needs the
 * context's level-1 block of SpMV entries to fit in shared memory (else
 * HBMC_ERR_INVALID_ARG).  Does not need hbmc_ic0.  Synchronizes.
 */
hbmc_status hbmc_sor(hbmc_ctx *ctx, const double *b_dev, double *x_dev, double omega, int32_t sweeps,
                     int32_t symmetric, double *relres);
/* The same on reordered vectors (length n_pad, HBMC order, dummies 0), with
 * no permutation and no residual; asynchronous on the context's stream. */
hbmc_status hbmc_sor_bar(hbmc_ctx *ctx, const double *b_dev, double *x_dev, double omega, int32_t sweeps,
                         int32_t symmetric);

/*
 * hbmc_spmv_dot_static - q = Abar p and p.q without allocating anything.
 *
 * The paper has no counterpart: this exists for callers that cannot
 * allocate device memory when they need the product: programs whose device
 * memory belongs entirely to another allocator (a framework's caching
 * allocator with a fixed budget, so a cudaMalloc of our own could fail or
 * fragment its pool), and time-critical loops that must not allocate after
 * start-up (cudaMalloc may synchronize the device).  It computes what the
 * solver's unsplit SpMV computes (same bits in q; with sell_split the
 * solver's product is the row-split one instead), but keeps its reduction scratch
 * in a fixed array of static device memory inside the library: 16 bytes plus
 * 8192 doubles (64 KiB) per device, held by every GPU that loads the library
 * until the process exits.
 *
 * p_dev, q_dev: device double[n_pad] in HBMC order (p may not alias q);
 * pq_dev: device double receiving p.q.  For an empty system (n = 0) only
 * pq_dev is used (set to 0; p_dev and q_dev may be NULL).  Asynchronous on
 * the context's stream.  Needs a context built with w = 32 and at most 32768 level-1
 * blocks (n_pad <= 32768 * bs * 32); larger contexts get
 * HBMC_ERR_INVALID_ARG with the limit in hbmc_last_error.  Calls no
 * cudaMalloc or cudaFree.  The first call on a device looks up the static
 * array's device address and sets a kernel attribute, so make that first
 * call before any stream capture begins.  All calls on a device share the
 * array: each clears it on its own stream before use, and calls whose
 * kernels could overlap on the GPU race, so order them (one stream, or
 * events).
 */
hbmc_status hbmc_spmv_dot_static(hbmc_ctx *ctx, const double *p_dev, double *q_dev, double *pq_dev);

/* ======================================================================
 * Batched solver: many independent SPD systems in one set of launches.
 *
 * Each system is blocked, colored and HBMC-ordered on its own (Sections
 * 4.1-4.2); the systems are then interleaved color by color, so one launch
 * per color sweeps the level-1 blocks of every system (Eq. "BAMC3": blocks
 * of one color are independent, and blocks of different systems never
 * couple).  Every system keeps its own CG scalars and its own stopping test;
 * its row arithmetic is the same as when it is solved alone.  w is 32.
 * ====================================================================== */

typedef struct hbmc_system {
  int64_t n;                /* host CSR of one system (conventions as hbmc_build) */
  const int64_t *row_ptr;
  const int32_t *col;
  const double *val;
  int32_t blocking;         /* HBMC_BLOCK_ALGEBRAIC or HBMC_BLOCK_BOXES */
  int64_t grid[3];          /* grid of this system for HBMC_BLOCK_BOXES */
} hbmc_system;

typedef struct hbmc_batch hbmc_batch; /* opaque */

/* Build a batch of nsys >= 1 systems with block size bs (w = 32).  opt may
 * be NULL; opt->box gives the box shape for systems that use box blocking;
 * opt->precision, loop_mode and device apply to the batch. */
hbmc_status hbmc_batch_build(int32_t nsys, const hbmc_system *systems, int32_t bs,
                             const hbmc_options *opt, hbmc_batch **out);
/* The same with w (Section 4.2's level-1 block width: w BMC blocks of a color
 * per level-1 block, w rows per SELL slice) 16 or 32; with w = 16 a warp
 * runs two level-1 blocks.  opt->sell_vslice > 0 gives the batch's SpMV the
 * variable-slice-height layout (same sums); row splitting is not supported.
 * hbmc_batch_features needs w = 32. */
hbmc_status hbmc_batch_build_w(int32_t nsys, const hbmc_system *systems, int32_t bs, int32_t w,
                               const hbmc_options *opt, hbmc_batch **out);
void hbmc_batch_destroy(hbmc_batch *b);
const char *hbmc_batch_last_error(const hbmc_batch *b);

/* Sizes: total unknowns (sum of n), padded rows, colors (max over systems),
 * level-1 blocks; any pointer may be NULL. */
hbmc_status hbmc_batch_info(const hbmc_batch *b, int64_t *n_total, int64_t *n_pad_total, int32_t *nc,
                            int64_t *units);
hbmc_status hbmc_batch_set_stream(hbmc_batch *b, void *stream);
hbmc_status hbmc_batch_set_precision(hbmc_batch *b, int32_t precision);

/* Shifted IC(0) of every system (Section 2, Eq. "ILU"; shift as in Section
 * 5.1) with its own shift: shifts[s] (host, NULL = all 0, each > -1).
 * bad_rows[s] (host, may be NULL) receives -1 or the first failing row of
 * system s in its own original numbering.  Returns HBMC_ERR_NOT_SPD_PIVOT if
 * any system failed; the others are factored and usable. */
hbmc_status hbmc_batch_ic0(hbmc_batch *b, const double *shifts, int64_t *bad_rows);

/* Solve every system to ||r_s|| / ||b_s|| < tol (Section 5.1 per system).
 * b_dev, x_dev: device doubles, the systems' vectors concatenated in order
 * (length sum of n); x_dev holds the initial guesses on entry.  Per-system
 * outputs (host arrays of nsys, each may be NULL): iterations, final
 * recurrence residual, true residual, status (an hbmc_status value), and
 * solve_ms: device time from the start of the solve until that system met
 * its tolerance.  Synchronizes.  Returns HBMC_OK when every system
 * converged, else the first non-OK per-system status. */
hbmc_status hbmc_batch_iccg(hbmc_batch *b, const double *b_dev, double *x_dev, double tol, int64_t maxit,
                            int64_t *iters, double *relres, double *true_relres, int32_t *status,
                            double *solve_ms);

/* Autotuner: builds the batch for each block size in bs_candidates (box
 * systems use the box shape of that size), factors with shift 0, solves b_dev
 * twice and keeps the faster size.  ms[k] (may be NULL) receives the timed
 * solve of candidate k (or -1 if it failed).  If cache_path is not NULL the
 * choice is stored there under a fingerprint of the systems' sizes and
 * reused without timing on the next call with the same fingerprint. */
hbmc_status hbmc_batch_autotune(int32_t nsys, const hbmc_system *systems, const int32_t *bs_candidates,
                                int32_t ncand, const hbmc_options *opt, const double *b_dev, double tol,
                                int64_t maxit, const char *cache_path, int32_t *best_bs, double *ms);
/* The same over every triple (bs_candidates[i], w_candidates[j],
 * vslice_candidates[k]): w 16 or 32; vslice 0 keeps the SpMV's SELL slice
 * height at w, K > 0 lets every slice take its height from {w, w/2, w/4}
 * (hbmc_options.sell_vslice = K).  ms[(i * nw + j) * nv + k] (may be NULL)
 * receives the timed solve of that triple or -1; *best_bs, *best_w,
 * *best_vslice the fastest.  The cache key includes the candidate lists. */
hbmc_status hbmc_batch_autotune_w(int32_t nsys, const hbmc_system *systems, const int32_t *bs_candidates,
                                  int32_t nbs, const int32_t *w_candidates, int32_t nw,
                                  const int32_t *vslice_candidates, int32_t nv, const hbmc_options *opt,
                                  const double *b_dev, double tol, int64_t maxit, const char *cache_path,
                                  int32_t *best_bs, int32_t *best_w, int32_t *best_vslice, double *ms);

/* Per-system feature vectors of a batch (host float[nsys *
 * HBMC_NUM_FEATURES], same definitions as hbmc_features). */
hbmc_status hbmc_batch_features(hbmc_batch *b, float *feat);

/* ======================================================================
 * Learned IC(0) shift.
 *
 * The paper's shifted ICCG (Section 5.1) sets the diagonal shift by hand.
 * Here the shift comes from a grid: shift c is 0 for c = 0 and 1e-3 * 2^(c-1)
 * for c = 1..HBMC_SHIFT_GRID-1.  The plain rule takes the first shift of the
 * grid whose IC(0) has only positive pivots.  A small MLP (D -> 32 -> 32 -> 1,
 * ReLU, inputs standardized) reads the matrix features plus the shift code
 * c / (HBMC_SHIFT_GRID - 1) and predicts log2 of the CG iterations that
 * shift would need; the learned choice is the grid shift with the lowest
 * prediction, with the plain rule as fallback when that factorization
 * fails.  Forward pass, gradients and Adam run in the library's kernels.
 * ====================================================================== */
#define HBMC_NUM_FEATURES 12
#define HBMC_SHIFT_GRID 13

/* Matrix features (host float[HBMC_NUM_FEATURES]), computed on the device over
 * the real rows of A: 0 log10 n; 1 mean nonzeros per row; 2 max nonzeros per
 * row; 3 min and 4 mean diagonal dominance a_ii / sum_{j!=i} |a_ij| (capped at
 * 10); 5 fraction of rows with dominance < 1 - 1e-9; 6 fraction of positive
 * off-diagonals; 7 mean and 8 standard deviation of log a_ii; 9 colors n_c;
 * 10 block size bs; 11 max dominance.  Needs w = 32. */
hbmc_status hbmc_features(hbmc_ctx *ctx, float *feat);

/* Shift c of the grid. */
double hbmc_shift_grid(int32_t c);

typedef struct hbmc_mlp hbmc_mlp; /* device-resident network and optimizer state */

/* Number of parameters for input width in_dim (layout: W1[32][D], b1[32],
 * W2[32][32], b2[32], w3[32], b3). */
int32_t hbmc_mlp_num_params(int32_t in_dim);
/* A network of in_dim inputs (1..256) on the current device, parameters all
 * zero, input standardization mean 0 and std 1 (set real ones with
 * hbmc_mlp_set_params).  *out receives it; the caller frees it with
 * hbmc_mlp_destroy.  INVALID_ARG for a bad in_dim or a NULL out, OOM when the
 * device memory cannot be had (then *out is NULL). */
hbmc_status hbmc_mlp_create(int32_t in_dim, hbmc_mlp **out);
/* Frees the network and its device memory; NULL is ignored. */
void hbmc_mlp_destroy(hbmc_mlp *net);
/* Message of the last failed call on net (NULL: of the last failed
 * hbmc_mlp_create). */
const char *hbmc_mlp_last_error(const hbmc_mlp *net);
/* Host parameters (NULL keeps the current ones) and input standardization
 * (mean, std > 0; NULL keeps them); resets the optimizer state. */
hbmc_status hbmc_mlp_set_params(hbmc_mlp *net, const float *params, const float *in_mean, const float *in_std);
hbmc_status hbmc_mlp_get_params(const hbmc_mlp *net, float *params);
/* out_dev[b] = network(X_dev[b][:]) for B samples (device floats, row-major). */
hbmc_status hbmc_mlp_forward(hbmc_mlp *net, const float *X_dev, int32_t B, float *out_dev);
/* Gradient of the loss L = mean_b (out_b - T_b)^2 with respect to every
 * parameter (device float[P]); *loss (host, may be NULL) receives L. */
hbmc_status hbmc_mlp_gradient(hbmc_mlp *net, const float *X_dev, const float *T_dev, int32_t B, float *grad_dev,
                              float *loss);
/* `steps` full-batch Adam steps (beta1 0.9, beta2 0.999, eps 1e-8) on L;
 * *loss (may be NULL) receives L after training. */
hbmc_status hbmc_mlp_train(hbmc_mlp *net, const float *X_dev, const float *T_dev, int32_t B, int32_t steps,
                           float lr, float *loss);
/* Learned shift for ctx's matrix: the grid shift with the lowest network
 * output (the predicted cost of each grid shift: log2 of its CG iterations
 * relative to the matrix's best, as learned_shift.py trains it); predicted
 * (host float[HBMC_SHIFT_GRID], may be NULL) gets the network's outputs.
 * Needs a network with in_dim = HBMC_NUM_FEATURES + 1. */
hbmc_status hbmc_predict_shift(hbmc_ctx *ctx, hbmc_mlp *net, double *shift, float *predicted);
/* Factor ctx with the learned shift (net != NULL) or the plain rule (net ==
 * NULL).  If the learned shift's IC(0) fails, the plain rule continues from
 * the next larger grid shift and *fallback is set to 1.  *shift_used gets the
 * shift that factored.  HBMC_ERR_NOT_SPD_PIVOT if no grid shift works. */
hbmc_status hbmc_ic0_auto(hbmc_ctx *ctx, hbmc_mlp *net, double *shift_used, int32_t *fallback);

#ifdef __cplusplus
}
#endif
#endif /* HBMC_H_ */

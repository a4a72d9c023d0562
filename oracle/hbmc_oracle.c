/*
 * Plain FP64 CPU oracle for HBMC-ordered IC(0)-CG.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The CUDA solver never
 * calls it and shares no code, header or table with it.
 *
 * Paper: T. Iwashita, S. Li, T. Fukaya, "Hierarchical Block Multi-Color
 * Ordering: A New Parallel Ordering Method for Vectorization and
 * Parallelization of the Sparse Triangular Solver in the ICCG Method"
 * (arXiv:1908.00741).
 *
 * What is computed here is the *definition* of the method's result: the
 * sequential IC(0)-CG solve of the explicitly reordered system
 * Abar = P A P^T (Section 3, Eq. "AB").  The HBMC level-1/level-2 block
 * structure (Section 4.2, Eqs. "BAMC1" to "y2-3") is only a parallel schedule
 * for this same sequential computation, so the oracle does not use it: every
 * factorization and substitution below runs row by row in index order.
 *
 * Rounding conventions (the paper is silent on them; these readings are
 * what the parity tests rely on):
 *   - every multiply-accumulate is one fused multiply-add, fma(), in the
 *     stated term order;
 *   - forward substitution and IC(0) sum their terms in ascending column
 *     order, backward substitution in descending column order (farthest
 *     column first in both cases); SpMV sums in ascending column order
 *     starting from zero;
 *   - dot products are either the plain left-to-right sum in the original
 *     index order (DOT_SEQUENTIAL) or the exactly rounded real dot product
 *     (DOT_EXACT), which does not depend on any order.
 * Build with -ffp-contract=off so that the compiler adds no other fusion.
 *
 * All indices are 0-based.  CSR matrices: row pointer int64[n+1], column
 * int32 sorted ascending within a row, values double.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* Blocking (Section 4.1; the blocking heuristic named in Section 5.1)       */
/* ------------------------------------------------------------------------ */

/* Geometric blocking of a lexicographic nx*ny*nz grid (x fastest) into boxes
 * of bx*by*bz points.  Box ids run lexicographically over the box grid (box x
 * index fastest).  Boxes cut by the grid edge keep only their in-grid points
 * and therefore hold fewer than bx*by*bz unknowns.  Returns the block count. */
ORC_API int64_t orc_blocks_boxes(int64_t nx, int64_t ny, int64_t nz, int64_t bx, int64_t by,
                                 int64_t bz, int64_t *block_of) {
  int64_t mx = (nx + bx - 1) / bx, my = (ny + by - 1) / by, mz = (nz + bz - 1) / bz;
  for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x)
        block_of[x + nx * (y + ny * z)] = (x / bx) + mx * ((y / by) + my * (z / bz));
  return mx * my * mz;
}

/* Algebraic blocking, Section 5.1: a new block is seeded with the unassigned
 * unknown of minimal number.  Growth rule (not stated in the paper; our
 * reading): repeatedly add the minimal-numbered unassigned unknown adjacent to
 * any current member until the block has bs members; if no adjacent unassigned
 * unknown is left, the block is closed short.  Blocks are numbered in creation
 * order.  Returns the block count. */
ORC_API int64_t orc_blocks_greedy(int64_t n, const int64_t *rp, const int32_t *ci, int64_t bs,
                                  int64_t *block_of) {
  for (int64_t i = 0; i < n; ++i) block_of[i] = -1;
  int64_t *cand = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int64_t *in_cand = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) in_cand[i] = -1;
  int64_t nblocks = 0, next_seed = 0;
  while (1) {
    while (next_seed < n && block_of[next_seed] >= 0) ++next_seed;
    if (next_seed == n) break;
    int64_t b = nblocks++;
    int64_t ncand = 0, size = 0;
    int64_t add = next_seed;
    while (1) {
      block_of[add] = b;
      ++size;
      if (size == bs) break;
      /* the new member's unassigned neighbours become candidates */
      for (int64_t e = rp[add]; e < rp[add + 1]; ++e) {
        int64_t j = ci[e];
        if (block_of[j] < 0 && in_cand[j] != b) {
          in_cand[j] = b;
          cand[ncand++] = j;
        }
      }
      /* pick the minimal-numbered candidate that is still unassigned */
      int64_t best = -1, best_pos = -1;
      for (int64_t t = 0; t < ncand; ++t)
        if (block_of[cand[t]] < 0 && (best < 0 || cand[t] < best)) {
          best = cand[t];
          best_pos = t;
        }
      if (best < 0) break;
      cand[best_pos] = cand[--ncand];
      add = best;
    }
  }
  free(cand);
  free(in_cand);
  return nblocks;
}

/* Greedy block coloring (Sections 4.1 and 5.1): two blocks are adjacent when
 * some a_ij != 0 joins a member of one to a member of the other.  Blocks are
 * visited in id order and each takes the smallest color not used by an
 * already colored adjacent block.  Returns the number of colors n_c. */
ORC_API int64_t orc_color_blocks(int64_t n, const int64_t *rp, const int32_t *ci, int64_t nblocks,
                                 const int64_t *block_of, int64_t *color) {
  /* members of each block, in ascending unknown number */
  int64_t *bptr = (int64_t *)calloc((size_t)nblocks + 1, sizeof(int64_t));
  int64_t *mem = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) bptr[block_of[i] + 1]++;
  for (int64_t b = 0; b < nblocks; ++b) bptr[b + 1] += bptr[b];
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nblocks + 1));
  memcpy(fill, bptr, sizeof(int64_t) * (size_t)nblocks);
  for (int64_t i = 0; i < n; ++i) mem[fill[block_of[i]]++] = i;
  free(fill);

  int64_t cap = 64, nc = 0;
  int64_t *used = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
  for (int64_t c = 0; c < cap; ++c) used[c] = -1;
  for (int64_t b = 0; b < nblocks; ++b) color[b] = -1;
  for (int64_t b = 0; b < nblocks; ++b) {
    for (int64_t t = bptr[b]; t < bptr[b + 1]; ++t) {
      int64_t i = mem[t];
      for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
        int64_t nb = block_of[ci[e]];
        if (nb != b && color[nb] >= 0) used[color[nb]] = b;
      }
    }
    int64_t c = 0;
    while (c < cap && used[c] == b) ++c;
    if (c == cap) {
      used = (int64_t *)realloc(used, sizeof(int64_t) * (size_t)(2 * cap));
      for (int64_t k = cap; k < 2 * cap; ++k) used[k] = -1;
      cap *= 2;
    }
    color[b] = c;
    if (c + 1 > nc) nc = c + 1;
  }
  free(used);
  free(bptr);
  free(mem);
  return nc;
}

/* ------------------------------------------------------------------------ */
/* Orderings: BMC and its HBMC secondary reordering (Section 4.2)            */
/* ------------------------------------------------------------------------ */

/* BMC order: colors ascending; inside a color, blocks by ascending id; inside
 * a block, members by ascending unknown number.  Padding (Section 4.2.1,
 * "dummy unknowns"): every block is padded to bs members with dummies at its
 * end and every color to a multiple of w blocks with all-dummy blocks, so each
 * color segment is a multiple of bs*w long.
 *
 * For the block at position p = k'*w + j (0-based) in color c and its l-th
 * member:
 *   BMC  (hbmc == 0):  pi = off_c + p*bs + l
 *   HBMC (hbmc != 0):  pi = off_c + k'*bs*w + l*w + j
 * HBMC takes, inside level-1 block k' (Eq. "simd-block": w consecutive BMC
 * blocks of one color), the first member of each of its w blocks, then the
 * second, and so on (the pick-up process of Section 4.2).
 *
 * Writes pi[n] and color_ptr[nc+1] (color c occupies [color_ptr[c],
 * color_ptr[c+1]) of the padded index space) and returns n_pad. */
ORC_API int64_t orc_ordering(int64_t n, int64_t nblocks, const int64_t *block_of,
                             const int64_t *color, int64_t nc, int64_t bs, int64_t w, int hbmc,
                             int64_t *pi, int64_t *color_ptr) {
  int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nblocks > 0 ? nblocks : 1));
  int64_t *cnt = (int64_t *)calloc((size_t)nc, sizeof(int64_t));
  for (int64_t b = 0; b < nblocks; ++b) pos[b] = cnt[color[b]]++;
  color_ptr[0] = 0;
  for (int64_t c = 0; c < nc; ++c) {
    int64_t nb_pad = (cnt[c] + w - 1) / w * w;
    color_ptr[c + 1] = color_ptr[c] + nb_pad * bs;
  }
  int64_t *member = (int64_t *)calloc((size_t)(nblocks > 0 ? nblocks : 1), sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) {
    int64_t b = block_of[i];
    int64_t c = color[b], p = pos[b], l = member[b]++;
    int64_t kp = p / w, j = p % w;
    pi[i] = hbmc ? color_ptr[c] + kp * bs * w + l * w + j : color_ptr[c] + p * bs + l;
  }
  free(pos);
  free(cnt);
  free(member);
  return color_ptr[nc];
}

/* Abar = P A P^T (Eq. "AB") on the padded index space: abar(pi(i), pi(j)) =
 * a(i, j), and every dummy row is an identity row (diagonal 1, no couplings).
 * Output CSR has n_pad rows, nnz(A) + (n_pad - n) entries, sorted columns. */
ORC_API void orc_permute(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                         const int64_t *pi, int64_t n_pad, int64_t *rp_out, int32_t *ci_out,
                         double *v_out) {
  int64_t *inv = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_pad > 0 ? n_pad : 1));
  for (int64_t k = 0; k < n_pad; ++k) inv[k] = -1;
  for (int64_t i = 0; i < n; ++i) inv[pi[i]] = i;
  rp_out[0] = 0;
  for (int64_t k = 0; k < n_pad; ++k) {
    int64_t i = inv[k];
    int64_t len = i < 0 ? 1 : rp[i + 1] - rp[i];
    rp_out[k + 1] = rp_out[k] + len;
  }
  for (int64_t k = 0; k < n_pad; ++k) {
    int64_t i = inv[k], o = rp_out[k];
    if (i < 0) {
      ci_out[o] = (int32_t)k;
      v_out[o] = 1.0;
      continue;
    }
    /* insertion sort of the relabelled row (rows are short) */
    int64_t len = rp[i + 1] - rp[i];
    for (int64_t t = 0; t < len; ++t) {
      int32_t c = (int32_t)pi[ci[rp[i] + t]];
      double a = v[rp[i] + t];
      int64_t s = t;
      while (s > 0 && ci_out[o + s - 1] > c) {
        ci_out[o + s] = ci_out[o + s - 1];
        v_out[o + s] = v_out[o + s - 1];
        --s;
      }
      ci_out[o + s] = c;
      v_out[o + s] = a;
    }
  }
  free(inv);
}

/* ------------------------------------------------------------------------ */
/* IC(0) factorization (Section 2, Eq. "ILU"; shifted form as used for the  */
/* Ieej test in Section 5.1)                                                 */
/* ------------------------------------------------------------------------ */

/* Incomplete Cholesky Abar ~= L L^T with L restricted to the pattern of the
 * lower triangle of Abar, and diagonal shift: the factored matrix has
 * diagonal (1 + shift) * abar_ii and the same off-diagonals.  Row by row in
 * index order:
 *   l_ij = (abar_ij - sum_{k<j} l_ik l_jk) / l_jj     for j < i in pattern(i),
 *          the sum running over k in pattern(i) and pattern(j), ascending k;
 *   l_ii = sqrt((1 + shift) abar_ii - sum_{k<i} l_ik^2), ascending k.
 * lval gets l_ij at the position of abar_ij for j < i (0 elsewhere); ldiag
 * gets l_ii and dinv 1 / l_ii.  Returns -1 on success, or the first row whose
 * pivot is not a positive finite number (the factorization stops there). */
ORC_API int64_t orc_ic0(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                        double shift, double *lval, double *ldiag, double *dinv) {
  const double scale = 1.0 + shift;
  for (int64_t e = 0; e < rp[n]; ++e) lval[e] = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double aii = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      int64_t j = ci[e];
      if (j == i) aii = v[e];
      if (j >= i) continue;
      double s = v[e];
      /* merge row i (columns < j, already computed) with row j (columns < j) */
      int64_t p = rp[i], q = rp[j];
      while (p < e && q < rp[j + 1] && ci[q] < j) {
        if (ci[p] == ci[q]) {
          s = fma(-lval[p], lval[q], s);
          ++p;
          ++q;
        } else if (ci[p] < ci[q]) {
          ++p;
        } else {
          ++q;
        }
      }
      lval[e] = s / ldiag[j];
    }
    double d = scale * aii;
    for (int64_t e = rp[i]; e < rp[i + 1] && ci[e] < i; ++e) d = fma(-lval[e], lval[e], d);
    if (!(d > 0.0) || !isfinite(d)) return i;
    ldiag[i] = sqrt(d);
    dinv[i] = 1.0 / ldiag[i];
  }
  return -1;
}

/* ------------------------------------------------------------------------ */
/* Substitutions (Section 2, Eqs. "for" and "back")                          */
/* ------------------------------------------------------------------------ */

/* Forward substitution y = L^{-1} r:
 *   y_i = (r_i - sum_{j<i} l_ij y_j) * dinv_i, terms in ascending j. */
ORC_API void orc_fwd(int64_t n, const int64_t *rp, const int32_t *ci, const double *lval,
                     const double *dinv, const double *r, double *y) {
  for (int64_t i = 0; i < n; ++i) {
    double s = r[i];
    for (int64_t e = rp[i]; e < rp[i + 1] && ci[e] < i; ++e) s = fma(-lval[e], y[ci[e]], s);
    y[i] = s * dinv[i];
  }
}

/* Position of entry (j, i) for every entry (i, j) of a structurally symmetric
 * CSR matrix (used to read column i of L as row i of U = L^T). */
ORC_API int orc_transpose_pos(int64_t n, const int64_t *rp, const int32_t *ci, int64_t *tpos) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      int64_t j = ci[e], lo = rp[j], hi = rp[j + 1];
      while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (ci[mid] < i) lo = mid + 1; else hi = mid;
      }
      if (lo == rp[j + 1] || ci[lo] != i) return 1; /* not structurally symmetric */
      tpos[e] = lo;
    }
  return 0;
}

/* Backward substitution z = U^{-1} y with U = L^T:
 *   z_i = (y_i - sum_{j>i} l_ji z_j) * dinv_i, terms in descending j. */
ORC_API void orc_bwd(int64_t n, const int64_t *rp, const int32_t *ci, const int64_t *tpos,
                     const double *lval, const double *dinv, const double *y, double *z) {
  for (int64_t i = n - 1; i >= 0; --i) {
    double s = y[i];
    for (int64_t e = rp[i + 1] - 1; e >= rp[i] && ci[e] > i; --e) s = fma(-lval[tpos[e]], z[ci[e]], s);
    z[i] = s * dinv[i];
  }
}

/* Sparse matrix-vector product q = A p, terms in ascending column order. */
ORC_API void orc_spmv(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                      const double *p, double *q) {
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) s = fma(v[e], p[ci[e]], s);
    q[i] = s;
  }
}

/* ------------------------------------------------------------------------ */
/* Row splitting of the SELL SpMV                                            */
/* ------------------------------------------------------------------------ */

/* Section 5.2.2: in SELL every row of a slice is padded to the slice's
 * longest row, so a slice whose row lengths are very unequal processes many
 * zeros (the paper counts 40% more processed elements than CRS on Audikw_1);
 * the remedy it proposes is to split the rows that are much longer than the
 * others.  Reading used here (the paper gives no rule): slices are the w
 * consecutive rows s*w .. s*w+w-1 of the padded Abar.  Slice s gets a head
 * width t_s in [1, max_r L_r] (L_r = row lengths) minimising
 *   cost(t) = w*t + sum_{r: L_r > t} ( (L_r - t) + cp * ceil((L_r - t) / P) ),
 * the largest t among equal costs: w*t stored head entries, every entry past
 * t once, plus cp per piece for writing and adding its partial sum.  Row r
 * keeps its first min(L_r, t_s) entries (ascending columns) as its head; the
 * rest is cut into pieces of P entries, the last one shorter.
 *
 * head[s] receives t_s.  The return value is the number of entries the split
 * layout processes: sum_s w*t_s for the heads plus the pieces as rows of
 * their own, sorted by length (longest first) and packed w to a slice, each
 * slice padded to its longest piece.  *nsplit and *npieces (may be NULL)
 * receive the number of split rows and of pieces. */
static int cmp_desc_i64(const void *a, const void *b) {
  const int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
  return (x < y) - (x > y);
}

ORC_API int64_t orc_split_plan(int64_t n_pad, const int64_t *rp, int32_t w, int32_t P, int32_t cp,
                               int32_t *head, int64_t *nsplit, int64_t *npieces) {
  const int64_t ns = n_pad / w;
  int64_t processed = 0, nsp = 0, npc = 0;
  for (int64_t s = 0; s < ns; ++s) {
    int64_t mx = 0;
    for (int32_t j = 0; j < w; ++j) {
      const int64_t len = rp[s * w + j + 1] - rp[s * w + j];
      if (len > mx) mx = len;
    }
    int64_t best_t = mx, best_c = -1;
    for (int64_t t = 1; t <= mx; ++t) {
      int64_t c = (int64_t)w * t;
      for (int32_t j = 0; j < w; ++j) {
        const int64_t len = rp[s * w + j + 1] - rp[s * w + j];
        if (len > t) c += (len - t) + (int64_t)cp * ((len - t + P - 1) / P);
      }
      if (best_c < 0 || c <= best_c) {
        best_c = c;
        best_t = t;
      }
    }
    head[s] = (int32_t)best_t;
    processed += (int64_t)w * best_t;
    for (int32_t j = 0; j < w; ++j) {
      const int64_t len = rp[s * w + j + 1] - rp[s * w + j];
      if (len > best_t) {
        ++nsp;
        npc += (len - best_t + P - 1) / P;
      }
    }
  }
  /* the pieces' lengths, longest first, w to a slice */
  int64_t *pl = (int64_t *)malloc(sizeof(int64_t) * (size_t)(npc > 0 ? npc : 1));
  int64_t k = 0;
  for (int64_t s = 0; s < ns; ++s)
    for (int32_t j = 0; j < w; ++j) {
      const int64_t len = rp[s * w + j + 1] - rp[s * w + j];
      for (int64_t a = head[s]; a < len; a += P) pl[k++] = (len - a < P) ? len - a : P;
    }
  qsort(pl, (size_t)npc, sizeof(int64_t), cmp_desc_i64);
  for (int64_t a = 0; a < npc; a += w) processed += (int64_t)w * pl[a];
  free(pl);
  if (nsplit) *nsplit = nsp;
  if (npieces) *npieces = npc;
  return processed;
}

/* q = A p with the rows cut as orc_split_plan cuts them: each part (the head,
 * then every piece) summed from zero in ascending column order with fma, and
 * the parts' sums added left to right: q_i = ((S_0 + S_1) + S_2) + ...
 * A row that is not cut gives exactly orc_spmv's value. */
ORC_API void orc_spmv_split(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, int32_t w,
                            const int32_t *head, int32_t P, const double *p, double *q) {
  for (int64_t i = 0; i < n; ++i) {
    const int64_t b = rp[i], e = rp[i + 1];
    int64_t cut = b + head[i / w];
    if (cut > e) cut = e;
    double acc = 0.0;
    for (int64_t k = b; k < cut; ++k) acc = fma(v[k], p[ci[k]], acc);
    for (int64_t a = cut; a < e; a += P) {
      const int64_t z = (a + P < e) ? a + P : e;
      double part = 0.0;
      for (int64_t k = a; k < z; ++k) part = fma(v[k], p[ci[k]], part);
      acc = acc + part;
    }
    q[i] = acc;
  }
}

/* ------------------------------------------------------------------------ */
/* Dot products                                                              */
/* ------------------------------------------------------------------------ */

enum { DOT_SEQUENTIAL = 0, DOT_EXACT = 1 };

/* Exactly rounded sum of a list of doubles: Shewchuk's non-overlapping
 * expansion (J. R. Shewchuk, "Adaptive precision floating-point arithmetic and
 * fast robust geometric predicates", 1997) kept as a growing list of partials,
 * then rounded once to nearest-even.  Non-finite inputs fall back to the plain
 * sum (which is then non-finite as well). */
typedef struct {
  double *p;
  int64_t len, cap;
  double plain;
} expansion;

static void exp_add(expansion *x, double v) {
  x->plain += v;
  int64_t k = 0;
  for (int64_t t = 0; t < x->len; ++t) {
    double y = x->p[t];
    if (fabs(v) < fabs(y)) { double tmp = v; v = y; y = tmp; }
    double hi = v + y;
    double lo = y - (hi - v);
    if (lo != 0.0) x->p[k++] = lo;
    v = hi;
  }
  if (k == x->cap) {
    x->cap *= 2;
    x->p = (double *)realloc(x->p, sizeof(double) * (size_t)x->cap);
  }
  x->p[k++] = v;
  x->len = k;
}

static double exp_round(const expansion *x) {
  if (!isfinite(x->plain)) return x->plain;
  int64_t t = x->len;
  if (t == 0) return 0.0;
  double hi = x->p[--t], lo = 0.0;
  while (t > 0) {
    double v = x->p[--t];
    double s = hi + v;
    lo = v - (s - hi);
    hi = s;
    if (lo != 0.0) break;
  }
  /* half-way case: the remaining partials decide the direction */
  if (t > 0 && ((lo < 0.0 && x->p[t - 1] < 0.0) || (lo > 0.0 && x->p[t - 1] > 0.0))) {
    double y = lo * 2.0;
    double s = hi + y;
    if (y == s - hi) hi = s;
  }
  return hi;
}

/* sum over idx[0..m) (or 0..m when idx is NULL) of a[k] * b[k]. */
ORC_API double orc_dot(int64_t m, const int64_t *idx, const double *a, const double *b, int mode) {
  if (mode == DOT_SEQUENTIAL) {
    double s = 0.0;
    for (int64_t t = 0; t < m; ++t) {
      int64_t k = idx ? idx[t] : t;
      s = fma(a[k], b[k], s);
    }
    return s;
  }
  expansion x;
  x.cap = 64;
  x.len = 0;
  x.plain = 0.0;
  x.p = (double *)malloc(sizeof(double) * (size_t)x.cap);
  for (int64_t t = 0; t < m; ++t) {
    int64_t k = idx ? idx[t] : t;
    double p = a[k] * b[k];
    double e = fma(a[k], b[k], -p); /* exact: a*b = p + e (no underflow) */
    exp_add(&x, p);
    if (e != 0.0) exp_add(&x, e);
  }
  double r = exp_round(&x);
  free(x.p);
  return r;
}

/* ------------------------------------------------------------------------ */
/* Preconditioned CG (IC(0)-CG, Section 2; stopping rule of Section 5.1)     */
/* ------------------------------------------------------------------------ */

/* Hestenes-Stiefel PCG on Abar xbar = bbar with M = L L^T:
 *   r = b - A x, z = M^{-1} r, p = z, rho = r.z
 *   repeat: q = A p; alpha = rho / (p.q); x += alpha p; r -= alpha q;
 *           stop when ||r||_2 / ||b||_2 < tol (iterations = number of x
 *           updates); z = M^{-1} r; rho' = r.z; p = z + (rho'/rho) p.
 * Vector updates are fma(alpha, p, x), fma(-alpha, q, r), fma(beta, p, z).
 * Dot products run over `order` (the n unknowns' positions in the padded
 * space, in original numbering order) with the given mode; dummies are zero
 * in every vector and contribute nothing.
 *
 * x is the initial guess on entry and the solution on exit.  hist (length
 * maxit+1, may be NULL) receives the relative residual after each iteration
 * (hist[0] for the initial guess).  Returns 0 when converged, 1 when maxit was
 * reached, 2 on breakdown (p.q or rho not positive and finite). */
/* The product q = A p of the iteration: plain, or with the rows cut by a
 * split plan (head != NULL); the initial residual always uses the plain one. */
typedef struct {
  int32_t w, P;
  const int32_t *head;
} split_spec;

static void loop_spmv(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const split_spec *sp,
                      const double *p, double *q) {
  if (sp && sp->head)
    orc_spmv_split(n, rp, ci, v, sp->w, sp->head, sp->P, p, q);
  else
    orc_spmv(n, rp, ci, v, p, q);
}

static int pcg_impl(int64_t n_pad, const int64_t *rp, const int32_t *ci, const double *v,
                    const double *lval, const double *dinv, const double *b, double *x,
                    int64_t m, const int64_t *order, int dot_mode, double tol, int64_t maxit,
                    int64_t *iters, double *relres, double *hist, const split_spec *sp) {
  int64_t *tpos = (int64_t *)malloc(sizeof(int64_t) * (size_t)(rp[n_pad] > 0 ? rp[n_pad] : 1));
  double *r = (double *)malloc(sizeof(double) * (size_t)n_pad);
  double *z = (double *)malloc(sizeof(double) * (size_t)n_pad);
  double *y = (double *)malloc(sizeof(double) * (size_t)n_pad);
  double *p = (double *)malloc(sizeof(double) * (size_t)n_pad);
  double *q = (double *)malloc(sizeof(double) * (size_t)n_pad);
  int status = 1;
  *iters = 0;
  if (orc_transpose_pos(n_pad, rp, ci, tpos)) {
    status = 3;
    goto done;
  }
  orc_spmv(n_pad, rp, ci, v, x, q);
  for (int64_t i = 0; i < n_pad; ++i) r[i] = b[i] - q[i];
  double bnorm = sqrt(orc_dot(m, order, b, b, dot_mode));
  if (bnorm == 0.0) {
    for (int64_t i = 0; i < n_pad; ++i) x[i] = 0.0;
    *relres = 0.0;
    if (hist) hist[0] = 0.0;
    status = 0;
    goto done;
  }
  double res = sqrt(orc_dot(m, order, r, r, dot_mode)) / bnorm;
  if (hist) hist[0] = res;
  *relres = res;
  if (res < tol) {
    status = 0;
    goto done;
  }
  orc_fwd(n_pad, rp, ci, lval, dinv, r, y);
  orc_bwd(n_pad, rp, ci, tpos, lval, dinv, y, z);
  for (int64_t i = 0; i < n_pad; ++i) p[i] = z[i];
  double rho = orc_dot(m, order, r, z, dot_mode);
  for (int64_t k = 1; k <= maxit; ++k) {
    if (!(rho > 0.0) || !isfinite(rho)) {
      status = 2;
      break;
    }
    loop_spmv(n_pad, rp, ci, v, sp, p, q);
    double pq = orc_dot(m, order, p, q, dot_mode);
    if (!(pq > 0.0) || !isfinite(pq)) {
      status = 2;
      break;
    }
    double alpha = rho / pq;
    for (int64_t i = 0; i < n_pad; ++i) {
      x[i] = fma(alpha, p[i], x[i]);
      r[i] = fma(-alpha, q[i], r[i]);
    }
    *iters = k;
    res = sqrt(orc_dot(m, order, r, r, dot_mode)) / bnorm;
    *relres = res;
    if (hist) hist[k] = res;
    if (res < tol) {
      status = 0;
      break;
    }
    if (k == maxit) break;
    orc_fwd(n_pad, rp, ci, lval, dinv, r, y);
    orc_bwd(n_pad, rp, ci, tpos, lval, dinv, y, z);
    double rho_new = orc_dot(m, order, r, z, dot_mode);
    double beta = rho_new / rho;
    for (int64_t i = 0; i < n_pad; ++i) p[i] = fma(beta, p[i], z[i]);
    rho = rho_new;
  }
done:
  free(tpos);
  free(r);
  free(z);
  free(y);
  free(p);
  free(q);
  return status;
}

ORC_API int orc_pcg(int64_t n_pad, const int64_t *rp, const int32_t *ci, const double *v,
                    const double *lval, const double *dinv, const double *b, double *x,
                    int64_t m, const int64_t *order, int dot_mode, double tol, int64_t maxit,
                    int64_t *iters, double *relres, double *hist) {
  return pcg_impl(n_pad, rp, ci, v, lval, dinv, b, x, m, order, dot_mode, tol, maxit, iters, relres, hist, NULL);
}

/* orc_pcg with q = A p of every iteration computed by orc_spmv_split (slice
 * height w, head widths head[n_pad / w], piece length P). */
ORC_API int orc_pcg_split(int64_t n_pad, const int64_t *rp, const int32_t *ci, const double *v,
                          const double *lval, const double *dinv, const double *b, double *x,
                          int64_t m, const int64_t *order, int dot_mode, double tol, int64_t maxit,
                          int64_t *iters, double *relres, double *hist, int32_t w, const int32_t *head,
                          int32_t P) {
  split_spec sp = {w, P, head};
  return pcg_impl(n_pad, rp, ci, v, lval, dinv, b, x, m, order, dot_mode, tol, maxit, iters, relres, hist, &sp);
}

/* ------------------------------------------------------------------------ */
/* SOR and symmetric SOR sweeps (Section 2: the iteration steps of the GS    */
/* and SOR methods are substitutions like those of IC(0); Section 3.1, Eq.   */
/* "xj": an equivalent reordering gives the same iterates).                  */
/*                                                                          */
/* On the reordered matrix, row by row in index order (forward sweep: i     */
/* ascending; the backward sweep of symmetric SOR: i descending):           */
/*   s   = sum_{j != i} abar_ij x_j    (ascending column, one fma per term,  */
/*                                      starting from zero)                  */
/*   t   = (b_i - s) * dinv_i,  dinv_i = 1 / abar_ii (the reciprocal, as in  */
/*                                      Fig. "C-vec"'s diaginv)               */
/*   x_i = fma(omega, t - x_i, x_i)                                          */
/* x is overwritten in place, so every x_j read is the newest value of row  */
/* j.  omega = 1 is Gauss-Seidel.  Returns 0, or 1 if a row has no diagonal */
/* entry or a zero one.                                                      */
/* ------------------------------------------------------------------------ */
static int sor_row(int64_t i, const int64_t *rp, const int32_t *ci, const double *v, const double *b, double *x,
                   double omega) {
  double s = 0.0, d = 0.0;
  for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
    if (ci[e] == i) d = v[e];
    else s = fma(v[e], x[ci[e]], s);
  }
  if (d == 0.0) return 1;
  const double t = (b[i] - s) * (1.0 / d);
  x[i] = fma(omega, t - x[i], x[i]);
  return 0;
}

ORC_API int orc_sor(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const double *b, double *x,
                    double omega, int64_t sweeps, int symmetric) {
  for (int64_t k = 0; k < sweeps; ++k) {
    for (int64_t i = 0; i < n; ++i)
      if (sor_row(i, rp, ci, v, b, x, omega)) return 1;
    if (symmetric)
      for (int64_t i = n - 1; i >= 0; --i)
        if (sor_row(i, rp, ci, v, b, x, omega)) return 1;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* ILU(0) and preconditioned BiCGStab for a nonsymmetric Abar whose pattern */
/* is symmetric (Section 2: IC(0)/ILU(0) preconditioning; the HBMC ordering  */
/* applies to ILU(0)'s substitutions as to IC(0)'s).                        */
/* ------------------------------------------------------------------------ */

/* ILU(0): Abar ~= L U, L unit lower with the pattern of the strict lower
 * triangle, U upper with the pattern of the upper triangle (diagonal scaled
 * by 1 + shift).  Row by row in index order, the row's entries in ascending
 * column j:
 *   w   = abar_ij - sum_{k < min(i,j)} l_ik u_kj   (k ascending, k in the row's
 *          pattern and in column j's; one fma per term)
 *   l_ij = w / u_jj  for j < i;   u_ij = w  for j >= i.
 * lval / uval get l_ij / u_ij at the position of abar_ij (0 elsewhere); udiag
 * gets u_ii and uinv 1 / u_ii.  tpos from orc_transpose_pos.  Returns -1, or
 * the first row whose pivot u_ii is zero or not finite (it stops there). */
ORC_API int64_t orc_ilu0(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, const int64_t *tpos,
                         double shift, double *lval, double *uval, double *udiag, double *uinv) {
  const double scale = 1.0 + shift;
  for (int64_t e = 0; e < rp[n]; ++e) {
    lval[e] = 0.0;
    uval[e] = 0.0;
  }
  for (int64_t i = 0; i < n; ++i) {
    int have_diag = 0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      const int64_t j = ci[e];
      const int64_t lim = j < i ? j : i;
      double s = j == i ? scale * v[e] : v[e];
      /* k < lim in row i and in row j (pattern symmetry: (k, j) in the
       * pattern iff k is a column of row j); u_kj sits at tpos of (j, k) */
      int64_t p = rp[i], q = rp[j];
      while (p < rp[i + 1] && ci[p] < lim && q < rp[j + 1] && ci[q] < lim) {
        if (ci[p] == ci[q]) {
          s = fma(-lval[p], uval[tpos[q]], s);
          ++p;
          ++q;
        } else if (ci[p] < ci[q]) {
          ++p;
        } else {
          ++q;
        }
      }
      if (j < i) {
        lval[e] = s / udiag[j];
      } else if (j == i) {
        if (s == 0.0 || !isfinite(s)) return i;
        udiag[i] = s;
        uinv[i] = 1.0 / s;
        have_diag = 1;
      } else {
        uval[e] = s;
      }
    }
    if (!have_diag) return i;
  }
  return -1;
}

/* Backward substitution with U: z_i = (y_i - sum_{j>i} u_ij z_j) * uinv_i,
 * terms in descending j (farthest column first, as for IC(0)). */
ORC_API void orc_bwd_u(int64_t n, const int64_t *rp, const int32_t *ci, const double *uval, const double *uinv,
                       const double *y, double *z) {
  for (int64_t i = n - 1; i >= 0; --i) {
    double s = y[i];
    for (int64_t e = rp[i + 1] - 1; e >= rp[i] && ci[e] > i; --e) s = fma(-uval[e], z[ci[e]], s);
    z[i] = s * uinv[i];
  }
}

/* z = (L U)^{-1} r: unit-lower forward substitution (orc_fwd with all-ones
 * dinv: y_i = (r_i - sum l_ij y_j) * 1), then orc_bwd_u. */
static void ilu_apply(int64_t n, const int64_t *rp, const int32_t *ci, const double *lval, const double *ones,
                      const double *uval, const double *uinv, const double *r, double *y, double *z) {
  orc_fwd(n, rp, ci, lval, ones, r, y);
  orc_bwd_u(n, rp, ci, uval, uinv, y, z);
}

/* Right-preconditioned BiCGStab (van der Vorst) on Abar with M = L U:
 *   r = b - A x, rh = r, rho_old = alpha = omega = 1, p = v = 0, rho = (rh, r)
 *   per iteration k:
 *     beta = (rho / rho_old) * (alpha / omega)
 *     p = r + beta (p - omega v)      [p_i = fma(beta, fma(-omega, v_i, p_i), r_i)]
 *     ph = M^{-1} p,  v = A ph,  alpha = rho / (rh, v)
 *     s = r - alpha v                 [fma(-alpha, v_i, r_i)]
 *     if ||s|| / ||b|| < tol: x = x + alpha ph [fma], stop (iteration k counted)
 *     sh = M^{-1} s,  t = A sh,  omega = (t, s) / (t, t)
 *     x = x + alpha ph + omega sh     [fma(omega, sh_i, fma(alpha, ph_i, x_i))]
 *     r = s - omega t                 [fma(-omega, t_i, s_i)]
 *     stop when ||r|| / ||b|| < tol (iteration k counted)
 *     rho_old = rho, rho = (rh, r)
 * Dots as in orc_pcg.  Returns 0 converged, 1 maxit, 2 breakdown (rho,
 * (rh, v), (t, t) or omega zero or not finite). */
ORC_API int orc_bicgstab(int64_t n_pad, const int64_t *rp, const int32_t *ci, const double *v, const double *lval,
                         const double *uval, const double *uinv, const double *b, double *x, int64_t m,
                         const int64_t *order, int dot_mode, double tol, int64_t maxit, int64_t *iters_out,
                         double *relres, double *hist) {
  double *r = calloc(n_pad, sizeof(double)), *rh = calloc(n_pad, sizeof(double));
  double *p = calloc(n_pad, sizeof(double)), *vv = calloc(n_pad, sizeof(double));
  double *s = calloc(n_pad, sizeof(double)), *t = calloc(n_pad, sizeof(double));
  double *ph = calloc(n_pad, sizeof(double)), *sh = calloc(n_pad, sizeof(double));
  double *y = calloc(n_pad, sizeof(double)), *ones = calloc(n_pad, sizeof(double));
  int status = 1;
  int64_t k = 0;
  for (int64_t i = 0; i < n_pad; ++i) ones[i] = 1.0;
  orc_spmv(n_pad, rp, ci, v, x, t);
  for (int64_t i = 0; i < n_pad; ++i) {
    r[i] = b[i] - t[i];
    rh[i] = r[i];
  }
  const double bnorm = sqrt(orc_dot(m, order, b, b, dot_mode));
  if (bnorm == 0.0) {
    for (int64_t i = 0; i < n_pad; ++i) x[i] = 0.0;
    *relres = 0.0;
    if (hist) hist[0] = 0.0;
    status = 0;
    goto done;
  }
  double res = sqrt(orc_dot(m, order, r, r, dot_mode)) / bnorm;
  if (hist) hist[0] = res;
  *relres = res;
  if (res < tol) {
    status = 0;
    goto done;
  }
  double rho_old = 1.0, alpha = 1.0, omega = 1.0;
  double rho = orc_dot(m, order, rh, r, dot_mode);
  for (k = 1; k <= maxit; ++k) {
    if (rho == 0.0 || !isfinite(rho)) {
      status = 2;
      --k;
      break;
    }
    const double beta = (rho / rho_old) * (alpha / omega);
    for (int64_t i = 0; i < n_pad; ++i) p[i] = fma(beta, fma(-omega, vv[i], p[i]), r[i]);
    ilu_apply(n_pad, rp, ci, lval, ones, uval, uinv, p, y, ph);
    orc_spmv(n_pad, rp, ci, v, ph, vv);
    const double rv = orc_dot(m, order, rh, vv, dot_mode);
    if (rv == 0.0 || !isfinite(rv)) {
      status = 2;
      --k;
      break;
    }
    alpha = rho / rv;
    for (int64_t i = 0; i < n_pad; ++i) s[i] = fma(-alpha, vv[i], r[i]);
    const double sres = sqrt(orc_dot(m, order, s, s, dot_mode)) / bnorm;
    if (sres < tol) { /* the half step already meets the tolerance */
      for (int64_t i = 0; i < n_pad; ++i) {
        x[i] = fma(alpha, ph[i], x[i]);
        r[i] = s[i];
      }
      if (hist) hist[k] = sres;
      *relres = sres;
      status = 0;
      break;
    }
    ilu_apply(n_pad, rp, ci, lval, ones, uval, uinv, s, y, sh);
    orc_spmv(n_pad, rp, ci, v, sh, t);
    const double tt = orc_dot(m, order, t, t, dot_mode);
    const double ts = orc_dot(m, order, t, s, dot_mode);
    if (!(tt > 0.0) || !isfinite(tt)) {
      status = 2;
      --k;
      break;
    }
    omega = ts / tt;
    for (int64_t i = 0; i < n_pad; ++i) {
      x[i] = fma(omega, sh[i], fma(alpha, ph[i], x[i]));
      r[i] = fma(-omega, t[i], s[i]);
    }
    res = sqrt(orc_dot(m, order, r, r, dot_mode)) / bnorm;
    if (hist) hist[k] = res;
    *relres = res;
    if (res < tol) {
      status = 0;
      break;
    }
    if (omega == 0.0 || !isfinite(omega)) {
      status = 2;
      break;
    }
    rho_old = rho;
    rho = orc_dot(m, order, rh, r, dot_mode);
  }
  if (k > maxit) k = maxit;
done:
  *iters_out = k;
  free(r);
  free(rh);
  free(p);
  free(vv);
  free(s);
  free(t);
  free(ph);
  free(sh);
  free(y);
  free(ones);
  return status;
}

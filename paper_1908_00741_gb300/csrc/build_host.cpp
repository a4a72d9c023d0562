// Host side of hbmc_build: CSR validation, BMC blocking and greedy block
// coloring (Sections 4.1 and 5.1), the HBMC secondary reordering with dummy
// padding (Section 4.2), Abar = P A P^T (Section 3, Eq. "AB"), and the packed
// device layouts (SELL with slice size w, Section 4.3.2).
#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstdio>
#include <functional>
#include <queue>
#include <utility>

#include "hbmc_internal.h"

namespace hbmc {
namespace {

bool fail(std::string &err, const char *msg, int64_t a = -1, int64_t b = -1) {
  char buf[256];
  if (a >= 0 && b >= 0)
    std::snprintf(buf, sizeof buf, "%s (row %lld, col %lld)", msg, (long long)a, (long long)b);
  else if (a >= 0)
    std::snprintf(buf, sizeof buf, "%s (%lld)", msg, (long long)a);
  else
    std::snprintf(buf, sizeof buf, "%s", msg);
  err = buf;
  return false;
}

// CSR checks: shape, sorted unique columns, positive diagonal, exact symmetry.
bool validate(int64_t n, const int64_t *rp, const int32_t *ci, const double *v, bool nonsym, std::string &err) {
  if (n < 0) return fail(err, "n < 0");
  if (n == 0) return true;
  if (!rp || !ci || !v) return fail(err, "null CSR pointer");
  if (n >= (int64_t(1) << 31) - 4096) return fail(err, "n too large for int32 column indices");
  if (rp[0] != 0) return fail(err, "row_ptr[0] != 0");
  for (int64_t i = 0; i < n; ++i)
    if (rp[i + 1] < rp[i]) return fail(err, "row_ptr decreases at row", i);
  for (int64_t i = 0; i < n; ++i) {
    bool diag = false;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      int64_t j = ci[e];
      if (j < 0 || j >= n) return fail(err, "column out of range", i, j);
      if (e > rp[i] && ci[e - 1] >= j) return fail(err, "columns not strictly ascending", i, j);
      if (j == i) {
        diag = true;
        if (nonsym ? (v[e] == 0.0 || !(v[e] < 1e308 && v[e] > -1e308))
                   : (!(v[e] > 0.0) || !(v[e] < 1e308)))
          return fail(err, nonsym ? "diagonal zero or not finite" : "diagonal not positive and finite", i);
      }
      if (!(v[e] == v[e]) || v[e] > 1e308 || v[e] < -1e308) return fail(err, "non-finite value", i, j);
    }
    if (!diag) return fail(err, "missing diagonal", i);
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      int64_t j = ci[e];
      if (j <= i) continue;
      const int32_t *lo = ci + rp[j], *hi = ci + rp[j + 1];
      const int32_t *f = std::lower_bound(lo, hi, (int32_t)i);
      if (f == hi || *f != i) return fail(err, "pattern not symmetric", i, j);
      if (!nonsym && v[rp[j] + (f - lo)] != v[e]) return fail(err, "values not symmetric", i, j);
    }
  return true;
}

// Geometric boxes over a lexicographic grid: box ids lexicographic over the
// box grid (box x index fastest).
int64_t blocks_boxes(const hbmc_options &o, std::vector<int64_t> &block_of) {
  const int64_t nx = o.grid[0], ny = o.grid[1], nz = o.grid[2];
  const int64_t bx = o.box[0], by = o.box[1], bz = o.box[2];
  const int64_t mx = (nx + bx - 1) / bx, my = (ny + by - 1) / by, mz = (nz + bz - 1) / bz;
  int64_t i = 0;
  for (int64_t z = 0; z < nz; ++z) {
    const int64_t kz = z / bz;
    for (int64_t y = 0; y < ny; ++y) {
      const int64_t ky = y / by;
      for (int64_t x = 0; x < nx; ++x, ++i) block_of[i] = x / bx + mx * (ky + my * kz);
    }
  }
  return mx * my * mz;
}

// Algebraic blocking of Section 5.1: a new block starts at the minimal-
// numbered unassigned unknown and grows by the minimal-numbered unassigned
// unknown adjacent to its members (min-heap of candidates) until it holds bs
// unknowns or no adjacent unassigned unknown is left.
int64_t blocks_algebraic(int64_t n, const int64_t *rp, const int32_t *ci, int32_t bs,
                         std::vector<int64_t> &block_of) {
  std::fill(block_of.begin(), block_of.end(), -1);
  std::vector<int64_t> seen(n, -1);  // block in which an unknown became a candidate
  std::priority_queue<int64_t, std::vector<int64_t>, std::greater<int64_t>> heap;
  int64_t nb = 0, seed = 0;
  for (;;) {
    while (seed < n && block_of[seed] >= 0) ++seed;
    if (seed == n) break;
    const int64_t b = nb++;
    while (!heap.empty()) heap.pop();
    int64_t next = seed;
    for (int32_t size = 1;; ++size) {
      block_of[next] = b;
      if (size == bs) break;
      for (int64_t e = rp[next]; e < rp[next + 1]; ++e) {
        const int64_t j = ci[e];
        if (block_of[j] < 0 && seen[j] != b) {
          seen[j] = b;
          heap.push(j);
        }
      }
      next = -1;
      while (!heap.empty()) {
        const int64_t c = heap.top();
        heap.pop();
        if (block_of[c] < 0) {
          next = c;
          break;
        }
      }
      if (next < 0) break;
    }
  }
  return nb;
}

// Greedy block coloring (Section 5.1), blocks visited in id order, each
// taking the smallest color unused by its already colored neighbours.
int32_t color_blocks(int64_t n, const int64_t *rp, const int32_t *ci, int64_t nb,
                     const std::vector<int64_t> &block_of, std::vector<int32_t> &color) {
  std::vector<int64_t> start(nb + 1, 0), members(n);
  for (int64_t i = 0; i < n; ++i) start[block_of[i] + 1]++;
  for (int64_t b = 0; b < nb; ++b) start[b + 1] += start[b];
  {
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for (int64_t i = 0; i < n; ++i) members[fill[block_of[i]]++] = i;
  }
  color.assign(nb, -1);
  std::vector<int64_t> taken;  // taken[c] == b: color c is used by a neighbour of b
  int32_t nc = 0;
  for (int64_t b = 0; b < nb; ++b) {
    for (int64_t t = start[b]; t < start[b + 1]; ++t) {
      const int64_t i = members[t];
      for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
        const int32_t c = color[block_of[ci[e]]];
        if (c >= 0) {
          if ((size_t)c >= taken.size()) taken.resize(c + 1, -1);
          taken[c] = b;
        }
      }
    }
    int32_t c = 0;
    while ((size_t)c < taken.size() && taken[c] == b) ++c;
    color[b] = c;
    nc = std::max(nc, c + 1);
  }
  return nc;
}

}  // namespace

// Variable slice height of the SpMV layout (the other remedy Section 5.2.2
// and the conclusions name for SELL's padding): each slice of w rows is cut
// into w / C sub-slices of C consecutive rows, C in {w, w/2, w/4} (C >= 1),
// each padded only to its own longest row.  The slice takes the C of least
// cost  sum over its sub-slices of C * (longest row) + cost * (w / C)
// (padded entries plus a per-sub-slice charge), the largest C among equal
// costs.  Rows keep their order (no sorting across rows: sigma = C); inside
// a sub-slice entry t of its row p sits at start + t * C + p.
hbmc_status plan_vslice(HostLayout &h, int32_t cost, std::string &err) {
  // Built from the SELL layout itself (a_ptr / a_col / a_val: a row's entries
  // first, then the guard column), so that it serves a batch's merged layout
  // as well as a single system's.
  const int32_t w = h.w;
  const int64_t ns = h.a_ptr.empty() ? 0 : (int64_t)h.a_ptr.size() - 1;
  const int64_t guard = h.n_pad;
  h.vslice_cost = cost;
  h.vs_c.assign(ns, (uint8_t)w);
  h.vs_first.assign(ns, 0);
  h.vs_ptr.assign(1, 0);
  std::vector<int64_t> len(w);
  for (int64_t s = 0; s < ns; ++s) {
    const int64_t width = (h.a_ptr[s + 1] - h.a_ptr[s]) / w;
    for (int32_t j = 0; j < w; ++j) {
      int64_t t = 0;
      while (t < width && h.a_col[h.a_ptr[s] + t * w + j] != guard) ++t;
      len[j] = t;
    }
    int32_t c_best = w;
    int64_t best = -1;
    for (int32_t C = w; C >= 1 && C >= w / 4; C /= 2) {
      if (w % C) break;
      int64_t c = (int64_t)cost * (w / C);
      for (int32_t k = 0; k < w / C; ++k) {
        int64_t mx = 0;
        for (int32_t j = k * C; j < (k + 1) * C; ++j) mx = std::max(mx, len[j]);
        c += (int64_t)C * mx;
      }
      if (best < 0 || c < best) {  // strictly less: ties keep the larger C
        best = c;
        c_best = C;
      }
      if (C == 1) break;
    }
    h.vs_c[s] = (uint8_t)c_best;
    h.vs_first[s] = (int64_t)h.vs_ptr.size() - 1;
    for (int32_t k = 0; k < w / c_best; ++k) {
      int64_t mx = 0;
      for (int32_t j = k * c_best; j < (k + 1) * c_best; ++j) mx = std::max(mx, len[j]);
      h.vs_ptr.push_back(h.vs_ptr.back() + mx * c_best);
    }
  }
  if ((int64_t)h.vs_ptr.size() - 1 >= INT32_MAX) {
    fail(err, "too many sub-slices", (int64_t)h.vs_ptr.size());
    return HBMC_ERR_INVALID_ARG;
  }
  h.vs_col.assign(h.vs_ptr.back(), (int32_t)guard);
  h.vs_val.assign(h.vs_ptr.back(), 0.0);
  for (int64_t s = 0; s < ns; ++s) {
    const int32_t C = h.vs_c[s];
    for (int32_t j = 0; j < w; ++j) {
      const int64_t sub = h.vs_first[s] + j / C;
      const int32_t p = j % C;
      for (int64_t t = 0; t < (h.a_ptr[s + 1] - h.a_ptr[s]) / w; ++t) {
        const int64_t src = h.a_ptr[s] + t * w + j;
        if (h.a_col[src] == guard) break;
        const int64_t slot = h.vs_ptr[sub] + t * C + p;
        h.vs_col[slot] = h.a_col[src];
        h.vs_val[slot] = h.a_val[src];
      }
    }
  }
  return HBMC_OK;
}

// Row splitting of the SpMV layout (Section 5.2.2: in SELL a slice's rows
// are padded to its longest row; the remedy is to split rows that are much
// longer than the others).  Slice s of w rows gets the head width t in
// [1, longest row] of least cost
//   w*t + sum over rows longer than t of (length - t) + cost * ceil((length - t) / P),
// the largest t among equal costs.  Each row keeps its first min(length, t)
// entries in the slice; the rest is cut into pieces of P entries (the last
// one shorter).  The pieces become rows of their own: sorted by length,
// longest first (ties by row, then piece), packed w to a slice.
hbmc_status plan_split(HostLayout &h, int32_t P, int32_t cost, std::string &err) {
  const int32_t w = h.w;
  if (w > 32) {
    fail(err, "row splitting needs w <= 32", w);
    return HBMC_ERR_INVALID_ARG;
  }
  const int64_t ns = h.n_pad / w;
  const int64_t guard = h.n_pad;
  h.split_piece = P;
  h.split_cost = cost;
  h.split_head.assign(ns, 0);
  h.sh_ptr.assign(ns + 1, 0);
  h.sl_mask.assign(ns, 0u);
  h.sl_first.assign(ns, 0);
  struct Piece {
    int64_t len, row, start;
  };
  std::vector<Piece> pieces;
  std::vector<int64_t> len(w);
  int64_t nsplit = 0;
  for (int64_t s = 0; s < ns; ++s) {
    int64_t mx = 0;
    for (int32_t j = 0; j < w; ++j) {
      len[j] = h.rp[s * w + j + 1] - h.rp[s * w + j];
      mx = std::max(mx, len[j]);
    }
    // cost(t) for every t; keep the last minimum
    int64_t t_best = mx, c_best = -1;
    for (int64_t t = 1; t <= mx; ++t) {
      int64_t c = (int64_t)w * t;
      for (int32_t j = 0; j < w; ++j) {
        const int64_t rest = len[j] - t;
        if (rest > 0) c += rest + (int64_t)cost * ((rest + P - 1) / P);
      }
      if (c_best < 0 || c <= c_best) {
        c_best = c;
        t_best = t;
      }
    }
    h.split_head[s] = (int32_t)t_best;
    h.sh_ptr[s + 1] = h.sh_ptr[s] + t_best * w;
    h.sl_first[s] = (int32_t)nsplit;
    for (int32_t j = 0; j < w; ++j) {
      if (len[j] <= t_best) continue;
      h.sl_mask[s] |= 1u << j;
      ++nsplit;
      const int64_t row = s * w + j;
      for (int64_t a = t_best; a < len[j]; a += P) pieces.push_back({std::min<int64_t>(P, len[j] - a), row, a});
    }
  }
  if (nsplit >= INT32_MAX || (int64_t)pieces.size() >= INT32_MAX) {
    fail(err, "too many split rows or pieces", (int64_t)pieces.size());
    return HBMC_ERR_INVALID_ARG;
  }
  h.split_rows = nsplit;
  h.split_pieces = (int64_t)pieces.size();
  // heads
  h.sh_col.assign(h.sh_ptr[ns], (int32_t)guard);
  h.sh_val.assign(h.sh_ptr[ns], 0.0);
  for (int64_t s = 0; s < ns; ++s)
    for (int32_t j = 0; j < w; ++j) {
      const int64_t row = s * w + j, b = h.rp[row];
      const int64_t e = std::min<int64_t>(h.rp[row + 1], b + h.split_head[s]);
      for (int64_t k = b; k < e; ++k) {
        const int64_t slot = h.sh_ptr[s] + (k - b) * w + j;
        h.sh_col[slot] = h.ci[k];
        h.sh_val[slot] = h.av[k];
      }
    }
  // pieces as rows, longest first; pieces were generated in (row, start) order
  std::vector<int64_t> order(pieces.size());
  for (size_t k = 0; k < order.size(); ++k) order[k] = (int64_t)k;
  std::stable_sort(order.begin(), order.end(),
                   [&](int64_t a, int64_t b) { return pieces[a].len > pieces[b].len; });
  const int64_t nv = (int64_t)(pieces.size() + w - 1) / w * w;
  const int64_t nts = nv / w;
  h.sp_ptr.assign(nts + 1, 0);
  for (int64_t k = 0; k < nts; ++k) h.sp_ptr[k + 1] = h.sp_ptr[k] + pieces[order[k * w]].len * w;
  h.sp_col.assign(h.sp_ptr[nts], (int32_t)guard);
  h.sp_val.assign(h.sp_ptr[nts], 0.0);
  std::vector<int32_t> slot_of(pieces.size());
  for (int64_t v = 0; v < (int64_t)order.size(); ++v) {
    const Piece &pc = pieces[order[v]];
    slot_of[order[v]] = (int32_t)v;
    const int64_t k = v / w, j = v % w, b = h.rp[pc.row] + pc.start;
    for (int64_t e = 0; e < pc.len; ++e) {
      const int64_t slot = h.sp_ptr[k] + e * w + j;
      h.sp_col[slot] = h.ci[b + e];
      h.sp_val[slot] = h.av[b + e];
    }
  }
  // the split rows' pieces, in row order then piece order (= generation order)
  h.cmb_ptr.assign(nsplit + 1, 0);
  h.cmb_slot.assign(pieces.size(), 0);
  int64_t r = -1, prev_row = -1;
  for (size_t k = 0; k < pieces.size(); ++k) {
    if (pieces[k].row != prev_row) {
      ++r;
      prev_row = pieces[k].row;
      h.cmb_ptr[r] = (int32_t)k;
    }
    h.cmb_slot[k] = slot_of[k];
  }
  h.cmb_ptr[nsplit] = (int32_t)pieces.size();
  return HBMC_OK;
}

// Per-unit records (see HostLayout) from the slice pointer arrays.
hbmc_status make_records(HostLayout &h, std::string &err) {
  const int32_t bs = h.bs;
  h.rec_ints = (8 + 2 * bs + 3) / 4 * 4;
  for (int kind = 0; kind < 3; ++kind) {
    const std::vector<int64_t> &op = kind == 0 ? h.fo_ptr : kind == 1 ? h.bo_ptr : h.a_ptr;
    const std::vector<int64_t> *ip = kind == 0 ? &h.fi_ptr : kind == 1 ? &h.bi_ptr : nullptr;
    std::vector<int32_t> &rec = kind == 0 ? h.rec_f : kind == 1 ? h.rec_b : h.rec_a;
    int64_t max_o = 0, max_i = 0;
    rec.assign((size_t)h.ntiles * h.rec_ints, 0);
    for (int64_t u = 0; u < h.ntiles; ++u) {
      int32_t *rc = rec.data() + (size_t)u * h.rec_ints;
      const int64_t s0 = u * bs;
      const int64_t ob = op[s0], olen = op[s0 + bs] - ob;
      const int64_t ib = ip ? (*ip)[s0] : 0, ilen = ip ? (*ip)[s0 + bs] - ib : 0;
      if (olen >= (int64_t(1) << 31) || ilen >= (int64_t(1) << 31)) {
        fail(err, "a level-1 block holds too many entries", u);
        return HBMC_ERR_INVALID_ARG;
      }
      max_o = std::max(max_o, olen);
      max_i = std::max(max_i, ilen);
      rc[0] = (int32_t)olen;
      rc[1] = (int32_t)ilen;
      rc[2] = (int32_t)(uint32_t)((uint64_t)ob & 0xffffffffu);
      rc[3] = (int32_t)(uint32_t)((uint64_t)ob >> 32);
      rc[4] = (int32_t)(uint32_t)((uint64_t)ib & 0xffffffffu);
      rc[5] = (int32_t)(uint32_t)((uint64_t)ib >> 32);
      for (int l = 0; l <= bs; ++l) {
        rc[6 + l] = (int32_t)(op[s0 + l] - ob);
        rc[7 + bs + l] = ip ? (int32_t)((*ip)[s0 + l] - ib) : 0;
      }
    }
    if (kind == 0) { h.max_o_f = max_o; h.max_i_f = max_i; }
    if (kind == 1) { h.max_o_b = max_o; h.max_i_b = max_i; }
    if (kind == 2) h.max_a = max_o;
  }
  return HBMC_OK;
}

hbmc_status build_host(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                       int32_t bs, int32_t w, const hbmc_options &opt, HostLayout &h,
                       std::string &err) {
  if (bs < 1 || bs > kMaxBs) {
    fail(err, "bs must be in [1, 64]", bs);
    return HBMC_ERR_INVALID_ARG;
  }
  if (!(w == 1 || w == 2 || w == 4 || w == 8 || w == 16 || w == 32)) {
    fail(err, "w must be 1, 2, 4, 8, 16 or 32", w);
    return HBMC_ERR_INVALID_ARG;
  }
  const bool nonsym = opt.nonsymmetric != 0;
  if (!validate(n, rp, ci, v, nonsym, err)) return HBMC_ERR_INVALID_ARG;
  if (opt.blocking == HBMC_BLOCK_BOXES) {
    if (opt.grid[0] < 1 || opt.grid[1] < 1 || opt.grid[2] < 1 ||
        opt.grid[0] * opt.grid[1] * opt.grid[2] != n) {
      fail(err, "box blocking: grid nx*ny*nz must equal n");
      return HBMC_ERR_INVALID_ARG;
    }
    if (opt.box[0] < 1 || opt.box[1] < 1 || opt.box[2] < 1 ||
        (int64_t)opt.box[0] * opt.box[1] * opt.box[2] != bs) {
      fail(err, "box blocking: bx*by*bz must equal bs");
      return HBMC_ERR_INVALID_ARG;
    }
  } else if (opt.blocking != HBMC_BLOCK_ALGEBRAIC) {
    fail(err, "unknown blocking rule", opt.blocking);
    return HBMC_ERR_INVALID_ARG;
  }

  h = HostLayout();
  h.nonsym = nonsym;
  h.n = n;
  h.bs = bs;
  h.w = w;
  h.nnz = n ? rp[n] : 0;

  // ---- blocking and coloring ------------------------------------------------
  h.block_of.assign(n, 0);
  h.nblocks = n == 0 ? 0
              : opt.blocking == HBMC_BLOCK_BOXES ? blocks_boxes(opt, h.block_of)
                                                 : blocks_algebraic(n, rp, ci, bs, h.block_of);
  h.nc = n ? color_blocks(n, rp, ci, h.nblocks, h.block_of, h.block_color) : 0;

  // ---- BMC order, padding and HBMC secondary reordering ---------------------
  // Block p-th in its color (ascending id) lands in level-1 block p / w at
  // lane p % w; its l-th member (ascending unknown number) goes to step l.
  std::vector<int64_t> cnt(h.nc, 0), pos(h.nblocks);
  for (int64_t b = 0; b < h.nblocks; ++b) pos[b] = cnt[h.block_color[b]]++;
  h.color_ptr.assign(h.nc + 1, 0);
  h.tile_ptr.assign(h.nc + 1, 0);
  for (int32_t c = 0; c < h.nc; ++c) {
    const int64_t tiles = (cnt[c] + w - 1) / w;
    h.tile_ptr[c + 1] = h.tile_ptr[c] + tiles;
    h.color_ptr[c + 1] = h.tile_ptr[c + 1] * bs * w;
  }
  h.ntiles = h.tile_ptr[h.nc];
  h.n_pad = h.color_ptr[h.nc];
  if (h.n_pad + kGuard >= (int64_t(1) << 31)) {
    fail(err, "padded size too large for int32 column indices", h.n_pad);
    return HBMC_ERR_INVALID_ARG;
  }
  h.pi.assign(n, 0);
  h.inv.assign(h.n_pad, -1);
  {
    std::vector<int32_t> member(h.nblocks, 0);
    for (int64_t i = 0; i < n; ++i) {
      const int64_t b = h.block_of[i];
      const int64_t p = pos[b], l = member[b]++;
      const int64_t k = h.color_ptr[h.block_color[b]] + (p / w) * bs * w + l * w + (p % w);
      h.pi[i] = k;
      h.inv[k] = (int32_t)i;
    }
  }

  // ---- Abar = P A P^T with identity dummy rows --------------------------------
  const int64_t np = h.n_pad;
  h.rp.assign(np + 1, 0);
  for (int64_t k = 0; k < np; ++k) {
    const int64_t i = h.inv[k];
    h.rp[k + 1] = h.rp[k] + (i < 0 ? 1 : rp[i + 1] - rp[i]);
  }
  h.ci.resize(h.rp[np]);
  h.av.resize(h.rp[np]);
  {
    std::vector<std::pair<int32_t, double>> row;
    for (int64_t k = 0; k < np; ++k) {
      const int64_t i = h.inv[k], o = h.rp[k];
      if (i < 0) {
        h.ci[o] = (int32_t)k;
        h.av[o] = 1.0;
        continue;
      }
      row.clear();
      for (int64_t e = rp[i]; e < rp[i + 1]; ++e) row.emplace_back((int32_t)h.pi[ci[e]], v[e]);
      std::sort(row.begin(), row.end(),
                [](const std::pair<int32_t, double> &a, const std::pair<int32_t, double> &b) {
                  return a.first < b.first;
                });
      for (size_t t = 0; t < row.size(); ++t) {
        h.ci[o + t] = row[t].first;
        h.av[o + t] = row[t].second;
      }
    }
  }

  // ---- strict lower CSR (IC(0) input) ----------------------------------------
  h.lrp.assign(np + 1, 0);
  h.adiag.assign(np, 0.0);
  for (int64_t k = 0; k < np; ++k) {
    int64_t c = 0;
    for (int64_t e = h.rp[k]; e < h.rp[k + 1]; ++e) {
      if (h.ci[e] < k) ++c;
      if (h.ci[e] == k) h.adiag[k] = h.av[e];
    }
    h.lrp[k + 1] = h.lrp[k] + c;
  }
  h.nnz_lower = h.lrp[np];
  h.lci.resize(h.nnz_lower);
  h.laval.resize(h.nnz_lower);
  h.l_to_abar.resize(h.nnz_lower);
  for (int64_t k = 0; k < np; ++k) {
    int64_t o = h.lrp[k];
    for (int64_t e = h.rp[k]; e < h.rp[k + 1] && h.ci[e] < k; ++e, ++o) {
      h.lci[o] = h.ci[e];
      h.laval[o] = h.av[e];
      h.l_to_abar[o] = e;
    }
  }
  if (nonsym) {
    // transposed values: lower entry (k, c) <- abar_ck (row c, column k > c)
    h.uaval.resize(h.nnz_lower);
    h.u_to_abar.resize(h.nnz_lower);
    for (int64_t k = 0; k < np; ++k)
      for (int64_t o = h.lrp[k]; o < h.lrp[k + 1]; ++o) {
        const int64_t c = h.lci[o];
        const int32_t *lo = h.ci.data() + h.rp[c], *hi = h.ci.data() + h.rp[c + 1];
        const int64_t e = h.rp[c] + (std::lower_bound(lo, hi, (int32_t)k) - lo);
        h.uaval[o] = h.av[e];
        h.u_to_abar[o] = e;
      }
    // upper rows: row i lists columns j > i ascending with the lower entry (j, i)
    h.urp.assign(np + 1, 0);
    for (int64_t i = 0; i < np; ++i) {
      int64_t c = 0;
      for (int64_t e = h.rp[i]; e < h.rp[i + 1]; ++e)
        if (h.ci[e] > i) ++c;
      h.urp[i + 1] = h.urp[i] + c;
    }
    h.uci.resize(h.urp[np]);
    h.upos.resize(h.urp[np]);
    for (int64_t i = 0; i < np; ++i) {
      int64_t f = h.urp[i];
      for (int64_t e = h.rp[i]; e < h.rp[i + 1]; ++e) {
        const int64_t j = h.ci[e];
        if (j <= i) continue;
        const int32_t *lo = h.lci.data() + h.lrp[j], *hi = h.lci.data() + h.lrp[j + 1];
        h.uci[f] = (int32_t)j;
        h.upos[f] = h.lrp[j] + (std::lower_bound(lo, hi, (int32_t)i) - lo);
        ++f;
      }
    }
  }

  // ---- SELL layouts, one slice per (level-1 block, step) ----------------------
  const int64_t nslices = np / w;
  const int64_t guard = np;  // padded slots gather index n_pad (always 0)
  const int64_t tile_rows = (int64_t)bs * w;

  // SpMV: all entries of each row, ascending columns.
  h.a_ptr.assign(nslices + 1, 0);
  for (int64_t s = 0; s < nslices; ++s) {
    int64_t len = 0;
    for (int32_t j = 0; j < w; ++j) {
      const int64_t k = s * w + j;
      len = std::max(len, h.rp[k + 1] - h.rp[k]);
    }
    h.a_ptr[s + 1] = h.a_ptr[s] + len * w;
  }
  h.a_col.assign(h.a_ptr[nslices], (int32_t)guard);
  h.a_val.assign(h.a_ptr[nslices], 0.0);
  for (int64_t s = 0; s < nslices; ++s)
    for (int32_t j = 0; j < w; ++j) {
      const int64_t k = s * w + j;
      for (int64_t e = h.rp[k], t = 0; e < h.rp[k + 1]; ++e, ++t) {
        const int64_t slot = h.a_ptr[s] + t * w + j;
        h.a_col[slot] = h.ci[e];
        h.a_val[slot] = h.av[e];
      }
    }

  if (opt.sell_split > 0) {
    const hbmc_status st = plan_split(h, opt.sell_split, opt.sell_split_cost > 0 ? opt.sell_split_cost : 2, err);
    if (st != HBMC_OK) return st;
  }
  if (opt.sell_vslice > 0) {
    const hbmc_status st = plan_vslice(h, opt.sell_vslice, err);
    if (st != HBMC_OK) return st;
  }

  // Forward (rows of L): other-color entries in ascending column order, then
  // same-block entries in ascending step.  Backward (rows of U = L^T):
  // other-color entries in descending column order, then same-block entries
  // in descending step.  Both orders put the column farthest from the
  // diagonal first.
  auto lower_index = [&](int64_t row, int64_t col) -> int64_t {
    const int32_t *lo = h.lci.data() + h.lrp[row], *hi = h.lci.data() + h.lrp[row + 1];
    const int32_t *f = std::lower_bound(lo, hi, (int32_t)col);
    return h.lrp[row] + (f - lo);
  };
  h.lmap_f.assign(h.nnz_lower, 0);
  h.lmap_b.assign(h.nnz_lower, 0);
  for (int dir = 0; dir < 2; ++dir) {
    std::vector<int64_t> &optr = dir == 0 ? h.fo_ptr : h.bo_ptr;
    std::vector<int64_t> &iptr = dir == 0 ? h.fi_ptr : h.bi_ptr;
    std::vector<int32_t> &ocol = dir == 0 ? h.fo_col : h.bo_col;
    std::vector<uint8_t> &im = dir == 0 ? h.fi_m : h.bi_m;
    std::vector<int64_t> &lmap = dir == 0 ? h.lmap_f : h.lmap_b;
    optr.assign(nslices + 1, 0);
    iptr.assign(nslices + 1, 0);
    // pass 1: slice lengths
    for (int64_t s = 0; s < nslices; ++s) {
      int64_t lo_max = 0, li_max = 0;
      const int64_t tile = s / bs, tbeg = tile * tile_rows, tend = tbeg + tile_rows;
      for (int32_t j = 0; j < w; ++j) {
        const int64_t k = s * w + j;
        int64_t lo = 0, li = 0;
        for (int64_t e = h.rp[k]; e < h.rp[k + 1]; ++e) {
          const int64_t c = h.ci[e];
          if (dir == 0 ? c >= k : c <= k) continue;
          if (c >= tbeg && c < tend) ++li; else ++lo;
        }
        lo_max = std::max(lo_max, lo);
        li_max = std::max(li_max, li);
      }
      optr[s + 1] = optr[s] + lo_max * w;
      iptr[s + 1] = iptr[s] + li_max * w;
    }
    ocol.assign(optr[nslices], (int32_t)guard);
    im.assign(iptr[nslices], 0);
    // pass 2: fill; padded same-block slots point at a step that is already
    // final when the slot is read (step 0 forward, step bs-1 backward)
    for (int64_t s = 0; s < nslices; ++s) {
      const int64_t tile = s / bs, tbeg = tile * tile_rows, tend = tbeg + tile_rows;
      const int64_t l = s % bs;
      for (int64_t t = iptr[s]; t < iptr[s + 1]; ++t) im[t] = (uint8_t)(dir == 0 ? 0 : bs - 1);
      for (int32_t j = 0; j < w; ++j) {
        const int64_t k = s * w + j;
        int64_t to = 0, ti = 0;
        const int64_t e0 = h.rp[k], e1 = h.rp[k + 1];
        for (int pass = 0; pass < 2; ++pass) {  // 0: other colors, 1: same block
          for (int64_t q = 0; q < e1 - e0; ++q) {
            const int64_t e = dir == 0 ? e0 + q : e1 - 1 - q;
            const int64_t c = h.ci[e];
            if (dir == 0 ? c >= k : c <= k) continue;
            const bool same = c >= tbeg && c < tend;
            if (same != (pass == 1)) continue;
            // lower entry holding this coefficient: (k, c) forward, (c, k) backward
            const int64_t le = dir == 0 ? lower_index(k, c) : lower_index(c, k);
            if (!same) {
              const int64_t slot = optr[s] + to * w + j;
              ocol[slot] = (int32_t)c;
              lmap[le] = slot;
              ++to;
            } else {
              const int64_t m = (c - tbeg) / w;
              if ((c - tbeg) % w != j || (dir == 0 ? m >= l : m <= l)) {
                fail(err, "internal: same-block coupling off its lane", k, c);
                return HBMC_ERR_INVALID_ARG;
              }
              const int64_t slot = iptr[s] + ti * w + j;
              im[slot] = (uint8_t)m;
              lmap[le] = -slot - 1;
              ++ti;
            }
          }
        }
      }
    }
  }

  // The same other-color entries without padding (loader-thread sweeps).
  const int64_t ntl = h.ntiles;
  for (int dir = 0; dir < 2; ++dir) {
    std::vector<int64_t> &xptr = dir == 0 ? h.fx_ptr : h.bx_ptr;
    std::vector<int32_t> &xrel = dir == 0 ? h.fx_rel : h.bx_rel;
    std::vector<int32_t> &xcol = dir == 0 ? h.fx_col : h.bx_col;
    std::vector<int64_t> &lmapx = dir == 0 ? h.lmapx_f : h.lmapx_b;
    int64_t &max_x = dir == 0 ? h.max_x_f : h.max_x_b;
    int64_t &max_row = dir == 0 ? h.max_xrow_f : h.max_xrow_b;
    const int64_t xstride = (tile_rows + 1 + 3) / 4 * 4;  // 16-byte rows of offsets
    xptr.assign(ntl + 1, 0);
    xrel.assign((size_t)ntl * xstride, 0);
    lmapx.assign(h.nnz_lower, -1);
    xcol.clear();
    for (int64_t u = 0; u < ntl; ++u) {
      const int64_t tbeg = u * tile_rows, tend = tbeg + tile_rows;
      int32_t *rel = xrel.data() + (size_t)u * xstride;
      int64_t len = 0;
      for (int64_t lr = 0; lr < tile_rows; ++lr) {
        const int64_t k = tbeg + lr;
        rel[lr] = (int32_t)len;
        const int64_t e0 = h.rp[k], e1 = h.rp[k + 1];
        int64_t rl = 0;
        for (int64_t q = 0; q < e1 - e0; ++q) {
          const int64_t e = dir == 0 ? e0 + q : e1 - 1 - q;
          const int64_t c = h.ci[e];
          if (dir == 0 ? c >= k : c <= k) continue;
          if (c >= tbeg && c < tend) continue;
          lmapx[dir == 0 ? lower_index(k, c) : lower_index(c, k)] = xptr[u] + len;
          xcol.push_back((int32_t)c);
          ++len;
          ++rl;
        }
        max_row = std::max(max_row, rl);
      }
      rel[tile_rows] = (int32_t)len;
      if (len >= (int64_t(1) << 31) - 32) {
        fail(err, "a level-1 block holds too many entries", u);
        return HBMC_ERR_INVALID_ARG;
      }
      const int64_t padded = (len + 31) / 32 * 32;
      xcol.resize(xptr[u] + padded, (int32_t)guard);
      xptr[u + 1] = xptr[u] + padded;
      max_x = std::max(max_x, padded);
    }
  }
  return make_records(h, err);
}

}  // namespace hbmc

// Host side of the batched solver: many independent SPD systems laid out as
// one block-diagonal system.
//
// Every system is blocked, colored and HBMC-ordered on its own (build_host).
// The batch then interleaves the systems color-major: color c of the batch
// holds color c of system 0, then of system 1, ...  A color sweep of the
// batch is therefore one launch over every system's level-1 blocks of that
// color (Eq. "BAMC3": level-1 blocks of one color are independent, and blocks
// of different systems never couple).  Inside a system the global order
// keeps the relative order of its unknowns, so every row's terms are summed in
// exactly the order the system alone would use.
#include <algorithm>
#include <cstdio>

#include "hbmc_internal.h"

namespace hbmc {
namespace {

void clear_vec(std::vector<int64_t> &v) { std::vector<int64_t>().swap(v); }

}  // namespace

hbmc_status build_batch_host(int32_t nsys, const hbmc_system *sys, int32_t bs, int32_t w,
                             const hbmc_options &opt, HostLayout &g, BatchMeta &meta, std::string &err) {
  if (nsys < 1 || !sys) {
    err = "batch: need at least one system";
    return HBMC_ERR_INVALID_ARG;
  }
  std::vector<HostLayout> H(nsys);
  meta = BatchMeta();
  meta.nsys = nsys;
  meta.n.assign(nsys, 0);
  meta.orig0.assign(nsys + 1, 0);
  meta.nc_sys.assign(nsys, 0);
  for (int32_t s = 0; s < nsys; ++s) {
    hbmc_options o = opt;
    o.blocking = sys[s].blocking;
    for (int k = 0; k < 3; ++k) o.grid[k] = sys[s].grid[k];
    std::string e;
    hbmc_status st = build_host(sys[s].n, sys[s].row_ptr, sys[s].col, sys[s].val, bs, w, o, H[s], e);
    if (st != HBMC_OK) {
      char buf[64];
      std::snprintf(buf, sizeof buf, "batch system %d: ", s);
      err = buf + e;
      return st;
    }
    // drop what the batch does not need
    std::vector<int32_t>().swap(H[s].ci);
    std::vector<double>().swap(H[s].av);
    clear_vec(H[s].rp);
    clear_vec(H[s].l_to_abar);
    clear_vec(H[s].block_of);
    meta.n[s] = H[s].n;
    meta.orig0[s + 1] = meta.orig0[s] + H[s].n;
    meta.nc_sys[s] = H[s].nc;
    meta.nc = std::max(meta.nc, H[s].nc);
  }
  const int32_t nc = meta.nc;
  const int64_t R = (int64_t)bs * w;

  // ---- global units, color-major --------------------------------------------
  std::vector<std::vector<int64_t>> gu(nsys);  // local unit -> global unit
  for (int32_t s = 0; s < nsys; ++s) gu[s].assign(H[s].ntiles, -1);
  meta.cu_start.assign((size_t)nsys * nc, 0);
  meta.cu_count.assign((size_t)nsys * nc, 0);
  g = HostLayout();
  g.bs = bs;
  g.w = w;
  g.nc = nc;
  g.tile_ptr.assign(nc + 1, 0);
  std::vector<std::pair<int32_t, int64_t>> owner;  // global unit -> (system, local unit)
  int64_t G = 0;
  for (int32_t c = 0; c < nc; ++c) {
    g.tile_ptr[c] = G;
    for (int32_t s = 0; s < nsys; ++s) {
      if (c >= H[s].nc) continue;
      meta.cu_start[(size_t)s * nc + c] = G;
      for (int64_t u = H[s].tile_ptr[c]; u < H[s].tile_ptr[c + 1]; ++u) {
        gu[s][u] = G++;
        owner.emplace_back(s, u);
        meta.unit_sys.push_back(s);
      }
      meta.cu_count[(size_t)s * nc + c] = G - meta.cu_start[(size_t)s * nc + c];
    }
  }
  g.tile_ptr[nc] = G;
  g.ntiles = G;
  g.n_pad = G * R;
  if (g.n_pad + kGuard >= (int64_t(1) << 31)) {
    err = "batch: padded size too large for int32 column indices";
    return HBMC_ERR_INVALID_ARG;
  }
  g.color_ptr.assign(nc + 1, 0);
  for (int32_t c = 0; c <= nc; ++c) g.color_ptr[c] = g.tile_ptr[c] * R;
  const int64_t N = g.n_pad;
  auto row_map = [&](int32_t s, int64_t k) -> int64_t { return gu[s][k / R] * R + k % R; };
  auto col_map = [&](int32_t s, int64_t c) -> int32_t {
    return (int32_t)(c == H[s].n_pad ? N : row_map(s, c));
  };

  // ---- sizes ------------------------------------------------------------------
  for (int32_t s = 0; s < nsys; ++s) {
    g.n += H[s].n;
    g.nnz += H[s].nnz;
    g.nnz_lower += H[s].nnz_lower;
    g.nblocks += H[s].nblocks;
  }

  // ---- slice-structured arrays --------------------------------------------------
  const int64_t nslices = G * bs;
  auto concat = [&](auto member_ptr, auto member_data, std::vector<int64_t> &gptr, auto &gdata,
                    bool map_cols) {
    gptr.assign(nslices + 1, 0);
    for (int64_t gu_id = 0; gu_id < G; ++gu_id) {
      const int32_t s = owner[gu_id].first;
      const int64_t u = owner[gu_id].second;
      const std::vector<int64_t> &lp = H[s].*member_ptr;
      for (int l = 0; l < bs; ++l) {
        const int64_t ls = u * bs + l, gs = gu_id * bs + l;
        gptr[gs + 1] = gptr[gs] + (lp[ls + 1] - lp[ls]);
      }
    }
    gdata.resize(gptr[nslices]);
    for (int64_t gu_id = 0; gu_id < G; ++gu_id) {
      const int32_t s = owner[gu_id].first;
      const int64_t u = owner[gu_id].second;
      const std::vector<int64_t> &lp = H[s].*member_ptr;
      const auto &ld = H[s].*member_data;
      for (int l = 0; l < bs; ++l) {
        const int64_t ls = u * bs + l, gs = gu_id * bs + l;
        for (int64_t t = 0; t < lp[ls + 1] - lp[ls]; ++t) {
          auto v = ld[lp[ls] + t];
          if (map_cols) v = (decltype(v))col_map(s, (int64_t)v);
          gdata[gptr[gs] + t] = v;
        }
      }
    }
  };
  concat(&HostLayout::a_ptr, &HostLayout::a_col, g.a_ptr, g.a_col, true);
  {
    // values follow the same slices
    g.a_val.resize(g.a_col.size());
    for (int64_t gu_id = 0; gu_id < G; ++gu_id) {
      const int32_t s = owner[gu_id].first;
      const int64_t u = owner[gu_id].second;
      for (int l = 0; l < bs; ++l) {
        const int64_t ls = u * bs + l, gs = gu_id * bs + l;
        std::copy(H[s].a_val.begin() + H[s].a_ptr[ls], H[s].a_val.begin() + H[s].a_ptr[ls + 1],
                  g.a_val.begin() + g.a_ptr[gs]);
      }
    }
  }
  concat(&HostLayout::fo_ptr, &HostLayout::fo_col, g.fo_ptr, g.fo_col, true);
  concat(&HostLayout::bo_ptr, &HostLayout::bo_col, g.bo_ptr, g.bo_col, true);
  concat(&HostLayout::fi_ptr, &HostLayout::fi_m, g.fi_ptr, g.fi_m, false);
  concat(&HostLayout::bi_ptr, &HostLayout::bi_m, g.bi_ptr, g.bi_m, false);

  // ---- strict lower CSR, diagonal, permutation ----------------------------------
  g.lrp.assign(N + 1, 0);
  g.adiag.assign(N, 0.0);
  g.inv.assign(N, -1);
  for (int64_t gu_id = 0; gu_id < G; ++gu_id) {
    const int32_t s = owner[gu_id].first;
    const int64_t u = owner[gu_id].second;
    for (int64_t r = 0; r < R; ++r) {
      const int64_t k = u * R + r, gr = gu_id * R + r;
      g.lrp[gr + 1] = H[s].lrp[k + 1] - H[s].lrp[k];
      g.adiag[gr] = H[s].adiag[k];
      g.inv[gr] = H[s].inv[k] >= 0 ? (int32_t)(meta.orig0[s] + H[s].inv[k]) : -1;
    }
  }
  for (int64_t r = 0; r < N; ++r) g.lrp[r + 1] += g.lrp[r];
  g.lci.resize(g.lrp[N]);
  g.laval.resize(g.lrp[N]);
  g.lmap_f.resize(g.lrp[N]);
  g.lmap_b.resize(g.lrp[N]);
  auto slot_map = [&](int32_t s, int64_t slot, const std::vector<int64_t> &lp_o,
                      const std::vector<int64_t> &lp_i, const std::vector<int64_t> &gp_o,
                      const std::vector<int64_t> &gp_i) -> int64_t {
    const bool in = slot < 0;
    const int64_t p = in ? -slot - 1 : slot;
    const std::vector<int64_t> &lp = in ? lp_i : lp_o;
    const int64_t ls = (int64_t)(std::upper_bound(lp.begin(), lp.end(), p) - lp.begin()) - 1;
    const int64_t gs = gu[s][ls / bs] * bs + ls % bs;
    const int64_t gslot = (in ? gp_i : gp_o)[gs] + (p - lp[ls]);
    return in ? -gslot - 1 : gslot;
  };
  for (int64_t gu_id = 0; gu_id < G; ++gu_id) {
    const int32_t s = owner[gu_id].first;
    const int64_t u = owner[gu_id].second;
    const HostLayout &h = H[s];
    for (int64_t r = 0; r < R; ++r) {
      const int64_t k = u * R + r, gr = gu_id * R + r;
      for (int64_t e = h.lrp[k], o = g.lrp[gr]; e < h.lrp[k + 1]; ++e, ++o) {
        g.lci[o] = (int32_t)row_map(s, h.lci[e]);
        g.laval[o] = h.laval[e];
        g.lmap_f[o] = slot_map(s, h.lmap_f[e], h.fo_ptr, h.fi_ptr, g.fo_ptr, g.fi_ptr);
        g.lmap_b[o] = slot_map(s, h.lmap_b[e], h.bo_ptr, h.bi_ptr, g.bo_ptr, g.bi_ptr);
      }
    }
  }
  g.pi.assign(g.n, 0);
  for (int32_t s = 0; s < nsys; ++s)
    for (int64_t i = 0; i < H[s].n; ++i) g.pi[meta.orig0[s] + i] = row_map(s, H[s].pi[i]);
  meta.n_pad.assign(nsys, 0);
  for (int32_t s = 0; s < nsys; ++s) meta.n_pad[s] = H[s].n_pad;
  return make_records(g, err);
}

}  // namespace hbmc

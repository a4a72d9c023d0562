// Dependency-driven substitution sweeps: every color of a sweep in one
// launch, with no barrier between colors.
//
// Section 4.3.3 counts n_c - 1 synchronizations per substitution: every
// level-1 block of color c waits for all of colors 1..c-1.  What a level-1
// block really needs is only the rows its other-color couplings read
// (Eq. "for3"), and those sit in a few level-1 blocks of earlier colors.  So
// here the synchronization is per level-1 block:
//   - each CUDA block takes a ticket from a monotonic counter; tickets run
//     through the level-1 blocks in sweep order (colors ascending for the
//     forward sweep, descending for the backward one), so a CUDA block only
//     ever waits on level-1 blocks whose tickets are smaller, i.e. owned by
//     CUDA blocks that started before it and are resident: the sweep makes
//     progress however many CUDA blocks fit on the GPU;
//   - before waiting it starts the bulk copies of everything its level-1
//     block reads that no other level-1 block of this sweep writes: record,
//     right-hand side, dinv, r (backward, for the fused r.z), the row offsets,
//     columns and coefficients of the other-color run and the same-block run;
//   - once they have landed, it gathers in rounds.  A row's other-color
//     terms are stored in sweep order (forward: ascending column, i.e.
//     earlier colors first; backward: descending), and the dependency list
//     is sorted the same way, so whatever prefix of the list is already
//     published covers a prefix of every row's terms.  Warp 0 polls the list
//     (acquire loads, bounded by %globaltimer) and publishes the first row
//     index that is not yet readable; every thread then adds its row's terms
//     up to that bound (L2 gathers, one thread per row, several in flight)
//     and the next round waits for the list to grow.  Only the terms of the
//     colors published last are left for the round after the final wait;
//   - it then runs the bs-step chains of Eqs. "y2-2" / "y2-3", stores its
//     rows and publishes its own epoch with a release store.
// The epoch of a launch is ticket / (level-1 blocks) + 1: every launch takes
// exactly one ticket per level-1 block, so counter and flags never need
// resetting.  Per-row term order and arithmetic are those of every other
// sweep kernel (other-color terms in the layout's order, then the same-block
// chain), so the results are bit-identical to them and to the oracle.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>
#include <vector>

#include "device_util.cuh"
#include "hbmc_internal.h"
#include "kernels.h"
#include "warp_common.cuh"

namespace hbmc {
namespace {

constexpr int kDagThreads = 256;
constexpr size_t kDagSmemBudget = 200 * 1024;
constexpr uint32_t kDagRecInts = 160;  // record of bs <= 64, rounded
constexpr uint32_t kDagRecOff = 16;    // record after the mbarrier
constexpr int kDagGather = 16;         // gathers in flight per thread
// A level-1 block that reads rows of more than this many level-1 blocks of
// one color waits for that whole color (one counter) instead of their flags.
constexpr int64_t kDagColorWait = 16;
constexpr int kDagChain = 4;  // same-block terms loaded together in a chain step
constexpr unsigned kDagPollCheck = 64;  // polls between looks at the abort word and the clock
// CUDA blocks per SM the register allocation leaves room for: 3 at up to 85
// registers a thread, 4 at up to 64.  The FP32 kernels fit 64 without
// spilling; the FP64 backward sweep would spill, so it keeps 3.  Shared
// memory may hold a launch to fewer (dag_occupancy).
template <typename T>
constexpr int dag_min_blocks() {
  return sizeof(T) == 4 ? 4 : 3;
}
constexpr int kDagAutoColors = 8;               // automatic selection: at least this many colors
constexpr uint32_t kDagAutoSmem = 110 * 1024;   // ... and two CUDA blocks per SM

template <typename T>
struct DagArgs {
  const int32_t *rec;      // per level-1 block records (same-block run)
  const int64_t *x_ptr;    // unpadded other-color runs: starts
  const int32_t *x_rel;    //   row offsets, x_stride ints per level-1 block
  const int32_t *x_col;
  const T *x_val;
  const uint8_t *i_m;
  const T *i_val;
  const T *dinv;
  const int32_t *order;    // ticket position -> level-1 block (nullptr: the same index)
  const int64_t *dep_ptr;  // per level-1 block: its dependency list
  const int32_t *dep;      //   v >= 0: level-1 block v; v < 0: every level-1 block of color -v-1
  const int32_t *unit_color;   // level-1 block -> color
  const int64_t *color_units;  // color -> its level-1 blocks
  const int64_t *color_first;  // color -> its first level-1 block (n_c + 1 entries)
  unsigned *flag;          // per level-1 block: epoch of its last published result
  unsigned *color_done;    // per color: level-1 blocks published in this launch
  const uint8_t *counted;  // per color: some level-1 block waits on its counter
  unsigned *exit_cnt;      // CUDA blocks of this launch that have finished
  unsigned long long *ticket;
  unsigned *abort;   // epoch of the last launch a wait of which ran out
  int64_t units;
  int nc;
  int64_t stall;     // test hook: this level-1 block never publishes (-1: none)
  int64_t lookahead; // tickets between a CUDA block and the one whose operands it prefetches into L2
  uint64_t wait_ns;  // bound of every wait
  int rec_ints, bs, x_stride;
  uint32_t off_xr, off_ts, off_tin, off_ds, off_rr, off_oc, off_vv, off_iv, off_im, off_pos;
};

// Gathers go through L1: the rows of a level-1 block share many columns (a
// compact block's neighbourhoods overlap), and a cached 32-byte sector only
// ever holds rows of one level-1 block that had published before it was
// read (every row of a level-1 block is written before its publication), so
// a cached copy is never stale.
template <typename G>
__device__ __forceinline__ G gather(const G *p) {
  return *p;
}

// Lane j's bs-step chain of a level-1 block (Eqs. "y2-2", "y2-3"; forward:
// steps ascending, backward: descending), each step's row stored as soon as
// it is final, with r.z for the backward sweep.  BS > 0: the step count is
// known at compile time and every step is unrolled, so the loads of the
// same-block coefficients and step indices (they do not depend on the chain)
// are issued ahead of it; a step then costs one round of shared-memory
// loads of earlier steps' results and its fused multiply-adds.  BS = 0: any
// bs, one step after another.
template <int BS, bool FWD, typename T, typename OUT>
__device__ __forceinline__ void dag_chain(int bs, const int32_t *__restrict__ i_rel, const T *__restrict__ iv,
                                          const uint8_t *__restrict__ im, T *__restrict__ ts,
                                          const T *__restrict__ ds, const double *__restrict__ rr, int j,
                                          OUT *__restrict__ out, float *__restrict__ out32, bool dot, double &rz) {
  if constexpr (BS > 0) {
    int rel[BS + 1];
#pragma unroll
    for (int l = 0; l <= BS; ++l) rel[l] = i_rel[l];
#pragma unroll
    for (int q = 0; q < BS; ++q) {
      const int l = FWD ? q : BS - 1 - q;
      // at most q same-block couplings (the steps already done)
      constexpr int kMax = BS - 1;
      T acc = ts[(l << 5) + j];
      const int p0 = rel[l] + j, pe = rel[l + 1];
      T v[kMax > 0 ? kMax : 1], g[kMax > 0 ? kMax : 1];
#pragma unroll
      for (int t = 0; t < kMax; ++t)
        if (t < q && p0 + 32 * t < pe) {
          v[t] = iv[p0 + 32 * t];
          g[t] = ts[(im[p0 + 32 * t] << 5) + j];
        }
#pragma unroll
      for (int t = 0; t < kMax; ++t)
        if (t < q && p0 + 32 * t < pe) acc = fma(-v[t], g[t], acc);
      const T yv = acc * ds[(l << 5) + j];
      ts[(l << 5) + j] = yv;
      out[(l << 5) + j] = (OUT)yv;
      if constexpr (!FWD && sizeof(T) == 4) out32[(l << 5) + j] = yv;
      if (!FWD && dot) rz = fma(rr[(l << 5) + j], (double)yv, rz);
    }
  } else {
    for (int q = 0; q < bs; ++q) {
      const int l = FWD ? q : bs - 1 - q;
      T acc = ts[(l << 5) + j];
      const int pe = i_rel[l + 1];
      for (int p = i_rel[l] + j; p < pe; p += 32 * kDagChain) {
        T v[kDagChain], g[kDagChain];
#pragma unroll
        for (int t = 0; t < kDagChain; ++t)
          if (p + 32 * t < pe) {
            v[t] = iv[p + 32 * t];
            g[t] = ts[(im[p + 32 * t] << 5) + j];
          }
#pragma unroll
        for (int t = 0; t < kDagChain; ++t)
          if (p + 32 * t < pe) acc = fma(-v[t], g[t], acc);
      }
      const T yv = acc * ds[(l << 5) + j];
      ts[(l << 5) + j] = yv;
      out[(l << 5) + j] = (OUT)yv;
      if constexpr (!FWD && sizeof(T) == 4) out32[(l << 5) + j] = yv;
      if (!FWD && dot) rz = fma(rr[(l << 5) + j], (double)yv, rz);
    }
  }
}

// Warp 0 (all 32 lanes) moves kd over the satisfied prefix of the
// dependency list [kd, kend): it ends at the first dependency whose rows are
// not all published in this launch (kend when every one is).  With `block`
// it waits until the prefix has grown (or is complete).  Returns false when
// the wait ran out (then it raises the launch's abort word and the solve's
// timeout) or another CUDA block of the launch gave up.
//
// The list is taken 32 entries at a time, one per lane; each lane keeps its
// entry's address and target in registers, so a poll is one load per lane
// (a per-block flag or a per-color counter), and the abort word and the
// clock are read only every kDagPollCheck polls.
template <typename T>
__device__ __forceinline__ bool dag_advance(const DagArgs<T> &a, int64_t &kd, int64_t kend, unsigned epoch,
                                            bool block, uint64_t deadline, int lane, Scalars *sc) {
  const int64_t k0 = kd;
  while (kd < kend) {
    const int64_t q = kd + lane;
    const unsigned *f = nullptr;
    unsigned target = 0;
    bool is_flag = true;
    if (q < kend) {
      const int32_t v = a.dep[q];
      is_flag = v >= 0;
      f = is_flag ? a.flag + v : a.color_done + (-v - 1);
      target = is_flag ? epoch : (unsigned)a.color_units[-v - 1];
    }
    for (unsigned spins = 1;; ++spins) {
      bool sat = true;
      if (f) {
        const unsigned x = ld_relaxed_gpu(f);
        sat = is_flag ? (int)(x - target) >= 0 : x >= target;
      }
      const unsigned m = __ballot_sync(0xffffffffu, sat);
      if (m == 0xffffffffu) {  // the whole window: go on with the next one
        kd = kd + 32 < kend ? kd + 32 : kend;
        break;
      }
      const int first = __ffs(~m) - 1;
      if (first > 0 || kd > k0 || !block) {
        kd += first;
        return true;
      }
      if (spins % kDagPollCheck == 0) {
        if (__any_sync(0xffffffffu, ld_relaxed_gpu(a.abort) == epoch)) return false;  // another CUDA block gave up
        if (__any_sync(0xffffffffu, global_ns() > deadline)) {
          if (lane == 0) {
            *(volatile unsigned *)a.abort = epoch;
            sc->timeout = 1;
            sc->done = 1;
          }
          return false;
        }
      }
    }
  }
  return true;
}

// The row bound that goes with the first unsatisfied dependency kd: forward,
// rows below it are readable (the dependency's first row); backward, rows
// from it on (the row after the dependency's last one).  All readable when
// the list is exhausted.
template <bool FWD, typename T>
__device__ __forceinline__ int64_t dag_bound(const DagArgs<T> &a, int64_t kd, int64_t kend, int64_t R) {
  if (kd >= kend) return FWD ? INT64_MAX : (int64_t)-1;
  const int32_t v = a.dep[kd];
  if (v >= 0) return (FWD ? (int64_t)v : (int64_t)v + 1) * R;
  const int c = -v - 1;
  return (FWD ? a.color_first[c] : a.color_first[c + 1]) * R;
}

// One level-1 block of a sweep.  Returns the ticket position k (>= 0) when
// the block's rows were computed and published, -1 when the CUDA block left
// early (the solve was already over, or a wait ran out).
template <int NT, int BS, bool FWD, typename T, typename IN, typename G, typename OUT>
__device__ __forceinline__ int64_t dag_unit(const DagArgs<T> &a, unsigned char *smem, const IN *in, const G *gsrc,
                                            OUT *out, float *out32, const double *r, Scalars *sc, bool check_done,
                                            bool dot, double &rz) {
  __shared__ unsigned long long s_ticket;
  __shared__ int s_done;
  __shared__ int64_t s_x[2];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  int32_t *rs = reinterpret_cast<int32_t *>(smem + kDagRecOff);
  int32_t *xr = reinterpret_cast<int32_t *>(smem + a.off_xr);
  T *ts = reinterpret_cast<T *>(smem + a.off_ts);
  IN *tin = reinterpret_cast<IN *>(smem + a.off_tin);  // == ts when IN is T
  T *ds = reinterpret_cast<T *>(smem + a.off_ds);
  double *rr = reinterpret_cast<double *>(smem + a.off_rr);
  int32_t *oc = reinterpret_cast<int32_t *>(smem + a.off_oc);
  T *vv = reinterpret_cast<T *>(smem + a.off_vv);
  T *iv = reinterpret_cast<T *>(smem + a.off_iv);
  uint8_t *im = smem + a.off_im;
  const int tid = threadIdx.x;
  // The ticket comes first and unconditionally, so that every launch takes
  // exactly `units` tickets whatever happens to it.
  if (tid == 0) {
    s_ticket = atomicAdd(a.ticket, 1ull);
    s_done = check_done ? *(volatile int *)&sc->done : 0;
  }
  __syncthreads();
  const unsigned long long t = s_ticket;
  const unsigned epoch = (unsigned)(t / (unsigned long long)a.units) + 1u;
  const int64_t k = (int64_t)(t % (unsigned long long)a.units);
  if (s_done) return -1;
  const int64_t u = a.order ? (int64_t)a.order[k] : k;
  const uint32_t R = (uint32_t)a.bs * 32u;
  const int64_t row0 = u * (int64_t)R;
  const uint32_t xbytes = (uint32_t)a.x_stride * 4u;
  // Copies of what no level-1 block of this sweep writes.
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
    mbar_expect_tx(bar, R * (uint32_t)(sizeof(IN) + sizeof(T)) + (dot ? R * 8u : 0u) + xbytes);
    tma_load_1d(tin, in + row0, R * (uint32_t)sizeof(IN), bar);
    tma_load_1d(ds, a.dinv + row0, R * (uint32_t)sizeof(T), bar);
    if (dot) tma_load_1d(rr, r + row0, R * 8u, bar);
    tma_load_1d(xr, a.x_rel + u * a.x_stride, xbytes, bar);
  }
  const int32_t *rc = a.rec + u * a.rec_ints;
  for (int q = tid; q < a.rec_ints; q += NT) rs[q] = rc[q];
  if (tid < 2) s_x[tid] = a.x_ptr[u + tid];
  __syncthreads();
  const int ilen = rs[1];
  const int64_t ibeg = rec64(rs, 4), xbeg = s_x[0];
  const uint32_t xlen = (uint32_t)(s_x[1] - s_x[0]);  // a multiple of 32 entries
  // The level-1 block one resident set of CUDA blocks later in the sweep
  // will get its slot when some block ahead of it leaves, typically as the
  // color before it completes, with its copies on the critical path: its
  // contiguous operands go to L2 now (a thread that is otherwise waiting).
  if (tid == 32 && k + a.lookahead < a.units) {
    const int64_t k2 = k + a.lookahead;
    const int64_t u2 = a.order ? (int64_t)a.order[k2] : k2;
    prefetch_l2(in + u2 * (int64_t)R, R * (uint32_t)sizeof(IN));
    prefetch_l2(a.dinv + u2 * (int64_t)R, R * (uint32_t)sizeof(T));
    const int64_t xb = a.x_ptr[u2], xe = a.x_ptr[u2 + 1];
    if (xe > xb) {
      prefetch_l2(a.x_col + xb, (uint32_t)(xe - xb) * 4u);
      prefetch_l2(a.x_val + xb, (uint32_t)(xe - xb) * (uint32_t)sizeof(T));
    }
  }
  if (tid == 0) {
    mbar_arrive_expect_tx(bar, xlen * (uint32_t)(4 + sizeof(T)) + (uint32_t)ilen * (uint32_t)(1 + sizeof(T)));
    if (xlen > 0) {
      tma_load_1d(oc, a.x_col + xbeg, xlen * 4u, bar);
      tma_load_1d(vv, a.x_val + xbeg, xlen * (uint32_t)sizeof(T), bar);
    }
    if (ilen > 0) {
      tma_load_1d(iv, a.i_val + ibeg, (uint32_t)ilen * (uint32_t)sizeof(T), bar);
      tma_load_1d(im, a.i_m + ibeg, (uint32_t)ilen, bar);
    }
  }
  // The first look at the dependency list overlaps the copies; later rounds
  // wait for it to grow.
  __shared__ int64_t s_bound[2];
  __shared__ int s_state[2];  // 1: every dependency published; 0: more to come; -1: give up
  const uint64_t deadline = global_ns() + a.wait_ns;
  int64_t kd = a.dep_ptr[u];
  const int64_t kend = a.dep_ptr[u + 1];
  if (tid < 32) {
    dag_advance<T>(a, kd, kend, epoch, false, deadline, tid, sc);  // does not wait, cannot fail
    __threadfence();  // acquire: the flags and counters read above before the gathers below
    if (tid == 0) {
      s_state[0] = kd >= kend ? 1 : 0;
      s_bound[0] = dag_bound<FWD, T>(a, kd, kend, (int64_t)R);
    }
  }
  const bool landed = mbar_wait(bar, 0, deadline);
  if (!__syncthreads_and(landed)) {
    if (tid == 0) {
      *(volatile unsigned *)a.abort = epoch;
      sc->timeout = 1;
      sc->done = 1;
      mbar_wait(bar, 0, deadline + a.wait_ns);  // let every copy land before the CUDA block leaves
    }
    __syncthreads();
    return -1;
  }
  int32_t *pos = reinterpret_cast<int32_t *>(smem + a.off_pos);
  for (int lr = tid; lr < (int)R; lr += NT) {
    ts[lr] = (T)tin[lr];
    pos[lr] = xr[lr];
  }
  for (int round = 0;; ++round) {
    if (round > 0) {
      if (tid < 32) {
        // the previous round took everything that was readable: wait for more
        const bool ok = dag_advance<T>(a, kd, kend, epoch, true, deadline, tid, sc);
        __threadfence();
        if (tid == 0) {
          s_state[round & 1] = ok ? (kd >= kend ? 1 : 0) : -1;
          s_bound[round & 1] = dag_bound<FWD, T>(a, kd, kend, (int64_t)R);
        }
      }
      // Double-buffered by round: a thread reads round r's entry after the
      // barrier that follows its writing, and warp 0 writes that entry again
      // only in round r + 2, after the barrier of round r + 1.
      __syncthreads();
    }
    const int st = s_state[round & 1];
    if (st < 0) return -1;  // every copy has landed
    const int64_t bound = s_bound[round & 1];
    // One thread per row (the same rows every round): the row's readable
    // other-color terms in the layout's order, kDagGather gathers in flight.
    for (int lr = tid; lr < (int)R; lr += NT) {
      int p = pos[lr];
      const int pe = xr[lr + 1];
      int pr = pe;  // the last round: every remaining term is readable
      if (st != 1) {
        pr = p;
        if constexpr (FWD) {
          while (pr < pe && (int64_t)oc[pr] < bound) ++pr;
        } else {
          while (pr < pe && (int64_t)oc[pr] >= bound) ++pr;
        }
      }
      if (pr == p) continue;
      T acc = ts[lr];
      for (; p < pr; p += kDagGather) {
        T g[kDagGather];
#pragma unroll
        for (int q = 0; q < kDagGather; ++q)
          if (p + q < pr) g[q] = (T)gather(gsrc + oc[p + q]);
#pragma unroll
        for (int q = 0; q < kDagGather; ++q)
          if (p + q < pr) acc = fma(-vv[p + q], g[q], acc);
      }
      ts[lr] = acc;
      pos[lr] = pr;
    }
    if (st == 1) break;
  }
  __syncthreads();
  // The chains on warp 0, then the publication.
  if (tid < 32) {
    dag_chain<BS, FWD, T, OUT>(a.bs, rs + 7 + a.bs, iv, im, ts, ds, rr, tid, out + row0,
                               out32 ? out32 + row0 : nullptr, dot, rz);
    __syncwarp();
    if (tid == 0 && u != a.stall) {
      __threadfence();  // release: the warp's stores (ordered by __syncwarp) before both publications
      st_relaxed_gpu(a.flag + u, epoch);
      const int c = a.unit_color[u];
      if (a.counted[c]) atomicAdd(a.color_done + c, 1u);
    }
  }
  return k;
}

// Every CUDA block, whichever way it leaves: the last one of the launch
// clears the per-color counters for the next launch (the kernel boundary
// orders the clearing before it).
template <typename T>
__device__ __forceinline__ void dag_exit(const DagArgs<T> &a) {
  if (threadIdx.x != 0) return;
  __threadfence();
  if (atomicAdd(a.exit_cnt, 1u) == (unsigned)(a.units - 1)) {
    for (int c = 0; c < a.nc; ++c) a.color_done[c] = 0u;
    *a.exit_cnt = 0u;
    __threadfence();
  }
}

template <typename T, typename Y, int BS>
__global__ void __launch_bounds__(kDagThreads, dag_min_blocks<T>())
    k_fwd_dag(const DagArgs<T> a, const double *__restrict__ r, Y *y, Scalars *sc, int check_done) {
  extern __shared__ __align__(128) unsigned char smem[];
  double rz = 0.0;
  dag_unit<kDagThreads, BS, true, T, double, Y, Y>(a, smem, r, y, y, nullptr, nullptr, sc, check_done != 0, false,
                                                   rz);
  dag_exit(a);
}

template <typename T, typename Y, int BS>
__global__ void __launch_bounds__(kDagThreads, dag_min_blocks<T>())
    k_bwd_dag(const DagArgs<T> a, const Y *__restrict__ yin, double *z, float *z32, const double *__restrict__ r,
              Scalars *sc, int check_done, int dot_mode, double *part) {
  extern __shared__ __align__(128) unsigned char smem[];
  double rz = 0.0;
  const int64_t k = dag_unit<kDagThreads, BS, false, T, Y, T, double>(
      a, smem, yin, zgather<T>(z, z32), z, sizeof(T) == 4 ? z32 : nullptr, r, sc, check_done != 0, dot_mode != 0, rz);
  // one partial per level-1 block, in sweep order; the last one reduces
  if (dot_mode && k >= 0) rz_partial(rz, sc, dot_mode, part, k, 1, a.units, (unsigned)a.units);
  dag_exit(a);
}

uint32_t a16(uint64_t v) { return (uint32_t)((v + 15) & ~uint64_t(15)); }

int x_stride_of(int bs, int w) { return (bs * w + 1 + 3) / 4 * 4; }

DagPlan plan_one(int bs, int w, bool fwd, int rec_ints, int64_t max_x, int64_t max_i, size_t tsize) {
  DagPlan p;
  const uint64_t R = (uint64_t)bs * w;
  p.off_xr = a16((uint64_t)kDagRecOff + (uint64_t)kDagRecInts * 4);
  p.off_ts = a16(p.off_xr + (uint64_t)x_stride_of(bs, w) * 4);
  uint64_t next = p.off_ts + R * tsize;
  p.off_tin = p.off_ts;
  if (fwd && tsize != 8) {
    p.off_tin = a16(next);
    next = p.off_tin + R * 8;
  }
  p.off_ds = a16(next);
  p.off_rr = a16(p.off_ds + R * tsize);
  p.off_oc = a16(p.off_rr + (fwd ? 0 : R * 8));
  p.off_vv = a16(p.off_oc + (uint64_t)max_x * 4);
  p.off_iv = a16(p.off_vv + (uint64_t)max_x * tsize);
  p.off_im = a16(p.off_iv + (uint64_t)max_i * tsize);
  p.off_pos = a16(p.off_im + (uint64_t)max_i);
  const uint64_t total = a16(p.off_pos + R * 4);
  p.smem_bytes = (uint32_t)std::min<uint64_t>(total, 0xffffffffu);
  p.ok = w == 32 && rec_ints <= (int)kDagRecInts && total <= kDagSmemBudget;
  return p;
}

const DagPlan &dag_plan(const DeviceLayout &d, bool fwd, int prec) {
  return prec == HBMC_PREC_F64 ? (fwd ? d.dg_f64_f : d.dg_f64_b) : (fwd ? d.dg_f32_f : d.dg_f32_b);
}

template <typename T>
DagArgs<T> dag_args(const DeviceLayout &d, bool fwd, const DagPlan &p) {
  DagArgs<T> a;
  a.rec = fwd ? d.rec_f : d.rec_b;
  a.rec_ints = d.rec_ints;
  a.x_ptr = fwd ? d.fx_ptr : d.bx_ptr;
  a.x_rel = fwd ? d.fx_rel : d.bx_rel;
  a.x_col = fwd ? d.fx_col : d.bx_col;
  a.x_stride = x_stride_of(d.bs, d.w);
  a.i_m = fwd ? d.fi_m : d.bi_m;
  if constexpr (sizeof(T) == 8) {
    a.x_val = (const T *)(fwd ? d.fx_val : d.bx_val);
    a.i_val = (const T *)(fwd ? d.fi_val : d.bi_val);
    a.dinv = (const T *)(fwd ? d.dinv : d.dinvb);
  } else {
    a.x_val = (const T *)(fwd ? d.fx_val32 : d.bx_val32);
    a.i_val = (const T *)(fwd ? d.fi_val32 : d.bi_val32);
    a.dinv = (const T *)(fwd ? d.dinv32 : d.dinvb32);
  }
  a.order = fwd ? nullptr : d.dag_order_b;
  a.dep_ptr = fwd ? d.dep_ptr_f : d.dep_ptr_b;
  a.dep = fwd ? d.dep_f : d.dep_b;
  a.flag = fwd ? d.dag_flag_f : d.dag_flag_b;
  a.unit_color = d.dag_unit_color;
  a.color_units = d.dag_color_units;
  a.color_first = d.tile_ptr_dev;
  a.color_done = fwd ? d.dag_color_done : d.dag_color_done + d.nc;
  a.counted = d.dag_counted + (fwd ? 0 : d.nc);
  a.exit_cnt = d.dag_exit + (fwd ? 0 : 1);
  a.nc = d.nc;
  a.ticket = d.dag_ticket + (fwd ? 0 : 1);
  a.abort = d.dag_abort + (fwd ? 0 : 1);
  a.units = d.nc > 0 ? d.tile_ptr[d.nc] : 0;
  a.stall = d.dag_stall;
  a.lookahead = (int64_t)d.sm_count * std::max(p.resident, 1);
  a.wait_ns = d.dag_wait_ns;
  a.bs = d.bs;
  a.off_xr = p.off_xr;
  a.off_ts = p.off_ts;
  a.off_tin = p.off_tin;
  a.off_ds = p.off_ds;
  a.off_rr = p.off_rr;
  a.off_oc = p.off_oc;
  a.off_vv = p.off_vv;
  a.off_iv = p.off_iv;
  a.off_im = p.off_im;
  a.off_pos = p.off_pos;
  return a;
}

template <typename K>
cudaError_t allow(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDagSmemBudget);
}

// Per level-1 block, what it waits for: the level-1 blocks holding the rows
// its other-color couplings read (the run's padding points past the last
// row and is skipped) -- except that where it reads more than kDagColorWait
// level-1 blocks of one color it waits for that whole color, entry
// -(color + 1): in a random input order a level-1 block reads a third of the
// level-1 blocks of each of several earlier colors, and one counter per
// color is far cheaper to poll than hundreds of flags.  The list is sorted
// in the order the row terms are stored (forward: by first row ascending;
// backward: by last row descending), so that a satisfied prefix of it makes
// a prefix of every row's terms readable.
void deps_of(const HostLayout &h, bool fwd, const std::vector<int64_t> &xp, const std::vector<int32_t> &xc,
             const std::vector<int32_t> &ucolor, std::vector<int64_t> &ptr, std::vector<int32_t> &dep) {
  const int64_t R = (int64_t)h.bs * h.w;
  ptr.assign((size_t)h.ntiles + 1, 0);
  dep.clear();
  std::vector<int64_t> mark((size_t)h.ntiles, -1);
  std::vector<int32_t> units, list;
  std::vector<int64_t> per_color((size_t)h.nc, 0);
  // sort key: the first level-1 block of an entry (forward), minus the one
  // after its last (backward)
  auto key = [&](int32_t v) -> int64_t {
    if (v >= 0) return fwd ? (int64_t)v : -((int64_t)v + 1);
    const int c = -v - 1;
    return fwd ? h.tile_ptr[c] : -h.tile_ptr[c + 1];
  };
  for (int64_t u = 0; u < h.ntiles; ++u) {
    units.clear();
    list.clear();
    for (int64_t e = xp[u]; e < xp[u + 1]; ++e) {
      const int64_t c = xc[(size_t)e];
      if (c < 0 || c >= h.n_pad) continue;
      const int64_t v = c / R;
      if (mark[(size_t)v] != u) {
        mark[(size_t)v] = u;
        units.push_back((int32_t)v);
      }
    }
    for (int32_t v : units) ++per_color[(size_t)ucolor[(size_t)v]];
    for (int c = 0; c < h.nc; ++c)
      if (per_color[(size_t)c] > kDagColorWait) list.push_back(-(c + 1));
    for (int32_t v : units)
      if (per_color[(size_t)ucolor[(size_t)v]] <= kDagColorWait) list.push_back(v);
    for (int32_t v : units) per_color[(size_t)ucolor[(size_t)v]] = 0;
    std::sort(list.begin(), list.end(), [&](int32_t x, int32_t y) { return key(x) < key(y); });
    dep.insert(dep.end(), list.begin(), list.end());
    ptr[(size_t)u + 1] = (int64_t)dep.size();
  }
}

}  // namespace

bool dag_host_tables(const HostLayout &h, DagTables &t) {
  t = DagTables();
  const size_t nx = (size_t)h.ntiles + 1;
  if (h.w != 32 || h.ntiles == 0 || h.fx_ptr.size() != nx || h.bx_ptr.size() != nx) return false;
  t.ucolor.assign((size_t)h.ntiles, 0);
  t.color_units.assign((size_t)h.nc, 0);
  for (int c = 0; c < h.nc; ++c) {
    t.color_units[(size_t)c] = h.tile_ptr[c + 1] - h.tile_ptr[c];
    for (int64_t u = h.tile_ptr[c]; u < h.tile_ptr[c + 1]; ++u) t.ucolor[(size_t)u] = c;
  }
  deps_of(h, true, h.fx_ptr, h.fx_col, t.ucolor, t.ptr_f, t.dep_f);
  deps_of(h, false, h.bx_ptr, h.bx_col, t.ucolor, t.ptr_b, t.dep_b);
  t.counted.assign(2 * (size_t)h.nc, 0);
  for (int dir = 0; dir < 2; ++dir)
    for (int32_t v : dir == 0 ? t.dep_f : t.dep_b)
      if (v < 0) t.counted[(size_t)dir * h.nc + (size_t)(-v - 1)] = 1;
  // backward sweep order: colors descending, level-1 blocks ascending within a color
  t.order_b.reserve((size_t)h.ntiles);
  for (int c = h.nc - 1; c >= 0; --c)
    for (int64_t u = h.tile_ptr[c]; u < h.tile_ptr[c + 1]; ++u) t.order_b.push_back((int32_t)u);
  return true;
}

void plan_dag_kernels(const HostLayout &h, DeviceLayout &d) {
  d.dg_f64_f = plan_one(h.bs, h.w, true, h.rec_ints, h.max_x_f, h.max_i_f, 8);
  d.dg_f64_b = plan_one(h.bs, h.w, false, h.rec_ints, h.max_x_b, h.max_i_b, 8);
  d.dg_f32_f = plan_one(h.bs, h.w, true, h.rec_ints, h.max_x_f, h.max_i_f, 4);
  d.dg_f32_b = plan_one(h.bs, h.w, false, h.rec_ints, h.max_x_b, h.max_i_b, 4);

}

template <int BS>
cudaError_t allow_bs() {
  cudaError_t e;
  if ((e = allow(k_fwd_dag<double, double, BS>)) || (e = allow(k_fwd_dag<float, float, BS>)) ||
      (e = allow(k_bwd_dag<double, double, BS>)) || (e = allow(k_bwd_dag<float, float, BS>)))
    return e;
  return cudaSuccess;
}

cudaError_t setup_dag_kernels() {
  cudaError_t e;
  if ((e = allow_bs<0>()) || (e = allow_bs<4>()) || (e = allow_bs<8>())) return e;
  return cudaSuccess;
}

template <int BS>
static cudaError_t occupancy_bs(DeviceLayout &d) {
  DagPlan *plans[4] = {&d.dg_f64_f, &d.dg_f64_b, &d.dg_f32_f, &d.dg_f32_b};
  const void *kernels[4] = {(const void *)k_fwd_dag<double, double, BS>, (const void *)k_bwd_dag<double, double, BS>,
                            (const void *)k_fwd_dag<float, float, BS>, (const void *)k_bwd_dag<float, float, BS>};
  for (int i = 0; i < 4; ++i) {
    plans[i]->resident = 0;
    if (!plans[i]->ok) continue;
    int blocks = 0;
    const cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernels[i], kDagThreads, plans[i]->smem_bytes);
    if (e != cudaSuccess) return e;
    plans[i]->resident = blocks;
  }
  return cudaSuccess;
}

cudaError_t dag_occupancy(DeviceLayout &d) {
  if (d.bs == 8) return occupancy_bs<8>(d);
  if (d.bs == 4) return occupancy_bs<4>(d);
  return occupancy_bs<0>(d);
}

bool dag_usable(const DeviceLayout &d, bool fwd, int prec) {
  return d.w == 32 && d.rec_f && d.dag_ticket && d.dag_color_done && d.tile_ptr_dev && (fwd ? d.dep_ptr_f : d.dep_ptr_b) &&
         (fwd || d.dag_order_b) && dag_plan(d, fwd, prec).ok;
}

// sweep_kernel 8 selects these for every sweep they can run.  Automatic
// selection (0) takes them for matrices with many colors, where the
// per-color launches pay a kernel boundary and a ramp per color, when at
// least two CUDA blocks fit on an SM.  Measured (GB300, bs 8, forward +
// backward sweep): 27-point 96^3 in a random order (23 colors) 0.37 ms
// against 0.55 ms per color in FP32, 0.54 against 0.89 ms in FP64; 3-DOF
// 100^3 (21 colors) 0.69 against 0.99 ms in FP32.  On the 7-point 128^3
// stencil (2 colors, short rows) the warp-per-level-1-block kernels are
// twice as fast and stay.
bool dag_selected(const DeviceLayout &d, int prec) {
  if (d.sweep_kernel != 0 && d.sweep_kernel != 8) return false;
  if (!dag_usable(d, true, prec) || !dag_usable(d, false, prec)) return false;
  if (d.sweep_kernel == 8) return true;
  const uint32_t most = std::max(dag_plan(d, true, prec).smem_bytes, dag_plan(d, false, prec).smem_bytes);
  return d.nc >= kDagAutoColors && most <= kDagAutoSmem;
}

template <int BS>
static void fwd_bs(const DeviceLayout &d, int prec, const double *r, bool check_done, cudaStream_t s, unsigned grid) {
  const DagPlan &p = dag_plan(d, true, prec);
  if (prec == HBMC_PREC_F64)
    k_fwd_dag<double, double, BS><<<grid, kDagThreads, p.smem_bytes, s>>>(dag_args<double>(d, true, p), r, d.y,
                                                                          d.sc, check_done ? 1 : 0);
  else
    k_fwd_dag<float, float, BS><<<grid, kDagThreads, p.smem_bytes, s>>>(dag_args<float>(d, true, p), r, d.y32,
                                                                        d.sc, check_done ? 1 : 0);
}

template <int BS>
static void bwd_bs(const DeviceLayout &d, int prec, const double *r, int dot_mode, bool check_done, cudaStream_t s,
                   unsigned grid) {
  const DagPlan &p = dag_plan(d, false, prec);
  if (prec == HBMC_PREC_F64)
    k_bwd_dag<double, double, BS><<<grid, kDagThreads, p.smem_bytes, s>>>(
        dag_args<double>(d, false, p), d.y, d.z, d.z32, r, d.sc, check_done ? 1 : 0, dot_mode, d.part);
  else
    k_bwd_dag<float, float, BS><<<grid, kDagThreads, p.smem_bytes, s>>>(
        dag_args<float>(d, false, p), d.y32, d.z, d.z32, r, d.sc, check_done ? 1 : 0, dot_mode, d.part);
}

void enqueue_fwd_dag(const DeviceLayout &d, int prec, const double *r, bool check_done, cudaStream_t s) {
  const int64_t units = d.nc > 0 ? d.tile_ptr[d.nc] : 0;
  if (units == 0) return;
  if (d.bs == 8) fwd_bs<8>(d, prec, r, check_done, s, (unsigned)units);
  else if (d.bs == 4) fwd_bs<4>(d, prec, r, check_done, s, (unsigned)units);
  else fwd_bs<0>(d, prec, r, check_done, s, (unsigned)units);
}

void enqueue_bwd_dag(const DeviceLayout &d, int prec, const double *r, int dot_mode, bool check_done,
                     cudaStream_t s) {
  const int64_t units = d.nc > 0 ? d.tile_ptr[d.nc] : 0;
  if (units == 0) return;
  if (d.bs == 8) bwd_bs<8>(d, prec, r, dot_mode, check_done, s, (unsigned)units);
  else if (d.bs == 4) bwd_bs<4>(d, prec, r, dot_mode, check_done, s, (unsigned)units);
  else bwd_bs<0>(d, prec, r, dot_mode, check_done, s, (unsigned)units);
}

}  // namespace hbmc

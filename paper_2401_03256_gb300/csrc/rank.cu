// rank.cu - the rank engine: Static, Naive-dynamic and Dynamic Frontier PageRank in one
// persistent cooperative kernel per call.
//
// Eq. 1 (Section 3.1) in pull form: R[v] = (1 - alpha)/n + sum_{u in in(v)} C[u] with the
// cached contribution C[u] = alpha R[u] / |out(u)| (Store<> gives the representation);
// in teleport mode a dead end's rank is spread over all vertices (+ alpha D / n, D = sum
// of the ranks of dead ends).
//
// Algorithm 1, synchronous form (Section 4.2):
//   phase 0   initial marking: every vertex of G^t.out(u) for each source u of the
//             pending changes, plus the deleted targets (= G^{t-1}.out(u) \ G^t.out(u)),
//             is set in the affected bitmap, stamped with the iteration it joins (0) and
//             appended to one of three lists by in-degree (thread / warp / block per
//             vertex).
//   iteration i: every affected vertex v reads ranks and contributions of parity i & 1
//             and writes parity (i + 1) & 1; |r - R[v]| feeds the L-inf max and, if it
//             exceeds tau_f, the out-neighbours of v are marked (stamped i + 1) and
//             appended, so they join in iteration i + 1.  A vertex scans its out-row at
//             most once per call: marks persist, so a second scan could not mark
//             anything new.  One grid barrier per iteration; all blocks read the same
//             L-inf value and stop together when it is <= tau.
//             Sparse iterations walk the affected lists; once they hold more than
//             n / dense_div vertices an iteration walks the sweep items of the affected
//             vertices in tier order (same set, better locality); marks made in dense
//             iterations are buffered per warp and appended to list 0 in runs.
//   writeback the final parity is copied to the other for every affected vertex (both
//             parities hold the current ranks between calls) and the per-call marks are
//             cleared.
// Static and Naive-dynamic run the same loop over all vertices without marking.
//
// Memory: column runs stream through L2 with evict-first priority, contributions are
// gathered and stored with evict-last priority so the contribution array stays in L2.
// Every value written by another block during the kernel (ranks, contributions, lists,
// stamps, per-iteration counters) is read with ld.global.cg (L2), never from a possibly
// stale L1.  The grid barrier's wait is bounded (globaltimer); on time-out the kernel
// records an error and every block returns.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "prdf_graph.cuh"

#include "rank_dev.cuh"

namespace prdf {

// In/out state of an out-of-line sweep of the sweep items (full and dense iterations).
template <bool F32>
struct SweepIo {
  const typename Store<F32>::R *Rin;
  const typename Store<F32>::C *Cin;
  typename Store<F32>::R *Rout;
  typename Store<F32>::C *Cout;
  const uint4 *T;
  uint32_t n0, n1, n2, off1, off2;
  uint32_t it, slot;
  uint32_t cnt[3];
  bool scan_all, expand;
  Iter<F32> I;
  const typename Store<F32>::R *s_base;
  unsigned long long *s_kmax;
  const uint8_t *s_active;
  WarpBuf *wb;
  Mass<F32> dacc;
  typename Num<F32>::B my_max;
  uint32_t my_v = 0, my_e = 0, my_xv = 0, my_xe = 0, my_app = 0;
};

// The three tiers of a full or dense iteration.
// MODE: 0 full sweeps (Static, Naive-dynamic), 1 Dynamic Frontier (expands in place),
// 2 continuation of a Dynamic Frontier call (only records the vertices to expand).
template <bool F32, int MODE>
__device__ __forceinline__ void sweep_tiers(const RankArgs<F32> &a, SweepIo<F32> &io) {
  constexpr bool DF = MODE == 1, CONT = MODE == 2;
  using S = Store<F32>;
  using R = typename S::R;
  using C = typename S::C;
  using B = typename Num<F32>::B;
  const uint32_t tid = threadIdx.x, lane = tid & 31;
  const uint32_t nwarps = (gridDim.x * kRankBlock) >> 5, gwarp = (blockIdx.x * kRankBlock + tid) >> 5;
  const bool multi = a.ncomp > 1;
  const R *Rin = io.Rin;
  const C *Cin = io.Cin;
  R *Rout = io.Rout;
  C *Cout = io.Cout;
  const uint4 *T = io.T;
  const uint32_t n0 = io.n0, n1 = io.n1, n2 = io.n2, off1 = io.off1, off2 = io.off2;
  const uint32_t it = io.it, slot = io.slot;
  const uint32_t cnt[3] = {io.cnt[0], io.cnt[1], io.cnt[2]};
  const bool scan_all = io.scan_all;
  const bool expand = (DF || CONT) && io.expand;
  const Iter<F32> I = io.I;
  Mass<F32> dacc = io.dacc;
  WarpBuf wb = *io.wb;
  B my_max = io.my_max;
  uint32_t my_v = 0, my_e = 0, my_xv = 0, my_xe = 0, my_app = 0;
  const unsigned long long pol_cols = l2_evict_first(), pol_c = l2_evict_last();

  auto live = [&](uint32_t v) -> bool { return !multi || io.s_active[__ldg(a.comp + v)]; };
  auto take = [&](uint32_t v) -> bool {
    return live(v) && (!scan_all || ldcg(a.stamp + v) <= (uint16_t)it);
  };
  auto finish_at = [&](uint32_t v, C sum, R rold, typename S::A ad) -> B {
    const uint32_t c = multi ? (uint32_t)__ldg(a.comp + v) : 0u;
    const B dr = finish_vertex(a, Rout, Cout, v, sum, rold, ad, I, dacc, pol_c, multi ? io.s_base[c] : a.base);
    if (multi) atomicMax(&io.s_kmax[c], Num<F32>::key(dr));
    else my_max = dr > my_max ? dr : my_max;
    return dr;
  };

    // tier 0: one thread per vertex, 32 consecutive items per warp
    for (uint32_t b0 = gwarp * 32; b0 < n0; b0 += nwarps * 32) {
      const uint32_t i = b0 + lane;
      int push = 0;
      uint32_t v = 0;
      if (i < n0 && take(ldcg(T + i).x)) {
        const uint4 item = ldcg(T + i);
        v = item.x;
        const R rold = ldcg(Rin + v);
        const typename S::A ad = __ldg(a.adeg + v);
        const uint32_t xw = expand ? __ldcg(a.xbits + (v >> 5)) : 0u;
        C sum = row_sum_thread(Cin, a.in_col + item.y, item.z, pol_cols, pol_c);
        B dr = finish_at(v, sum, rold, ad);
        my_v++;
        my_e += item.z;
        push = expand && dr > a.ftol && first_expansion_pre(a.xbits, v, xw);
      }
      if constexpr (DF) {
        if (expand) queue_expansion(a, push, v, lane, wb);
      }
      if constexpr (CONT) record_expansion(a, push, v, lane, slot);
    }

    // tier 1: rows of lo < len <= group_max by 8-lane groups, four vertices per warp
    {
      const uint32_t grp = lane >> 3, gl = lane & 7;
      for (uint32_t b0 = gwarp * 4; b0 < n1; b0 += nwarps * 4) {
        const uint32_t i = b0 + grp;
        const bool act = i < n1 && take(ldcg(T + off1 + i).x);
        uint32_t xw = 0;
        uint4 item = make_uint4(0, 0, 0, 0);
        R rold = (R)0;
        typename S::A ad = (typename S::A)0;
        C sum = (C)0;
        if (act) {
          item = ldcg(T + off1 + i);
          if (gl == 0) {
            rold = ldcg(Rin + item.x);
            ad = __ldg(a.adeg + item.x);
            if (expand) xw = __ldcg(a.xbits + (item.x >> 5));
          }
          const uint32_t *cols = a.in_col + item.y;
          uint4 q[2];
#pragma unroll
          for (int r = 0; r < 2; r++) {
            const uint32_t j = 4 * (gl + 8 * r);
            if (j < item.z) q[r] = ld_cols(cols + j, pol_cols);
          }
#pragma unroll
          for (int r = 0; r < 2; r++) {
            const uint32_t j = 4 * (gl + 8 * r);
            if (j < item.z) sum += gather4(Cin, q[r], min(4u, item.z - j), pol_c);
          }
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
        int push = 0;
        if (act && gl == 0) {
          B dr = finish_at(item.x, sum, rold, ad);
          my_v++;
          my_e += item.z;
          push = expand && dr > a.ftol && first_expansion_pre(a.xbits, item.x, xw);
        }
        if constexpr (DF) {
          if (expand) queue_expansion(a, push, item.x, lane, wb);
        }
        if constexpr (CONT) record_expansion(a, push, item.x, lane, slot);
      }
    }

    // tier 2: chunks of chunk_len edges dealt round-robin to warps (a hub's consecutive chunks
    // land on different warps); a row split into several chunks is finished by the warp
    // that completes its last chunk, which adds the partial sums in chunk order
    C *part = a.partials;
    for (uint32_t k = gwarp; k < n2; k += nwarps) {
      const uint4 ch = ldcg(T + off2 + k);
      const uint32_t v = ch.x;
      if (!take(v)) continue;
      const uint32_t len = ch.z & 0x3FFu;
      const bool multi = (ch.z >> 31) != 0;
      R rold = (R)0;
      typename S::A ad = (typename S::A)0;
      uint32_t deg = len, xw = 0;
      if (lane == 0) {
        rold = ldcg(Rin + v);
        ad = __ldg(a.adeg + v);
        if (multi) deg = __ldg(&a.in_rd[v]).y;
        if (expand) xw = __ldcg(a.xbits + (v >> 5));
      }
      const uint32_t *cols = a.in_col + ch.y;
      uint4 q[4];
#pragma unroll
      for (int r = 0; r < 4; r++) {
        const uint32_t j = 4 * (lane + 32 * r);
        if (j < len) q[r] = ld_cols(cols + j, pol_cols);
      }
      C sum = (C)0;
#pragma unroll
      for (int r = 0; r < 4; r++) {
        const uint32_t j = 4 * (lane + 32 * r);
        if (j < len) sum += gather4(Cin, q[r], min(4u, len - j), pol_c);
      }
      sum = warp_sum(sum);
      int finish = 1;
      if (multi) {
        // publish this chunk's partial; the last of the row's chunks adds them up
        const uint32_t nch = (__shfl_sync(kFull, deg, 0) + a.chunk - 1) / a.chunk;
        uint32_t old = 0;
        if (lane == 0) {
          part[ch.w] = sum;
          __threadfence();
          old = atomicAdd(&a.chunk_done[v], 1u);
        }
        old = __shfl_sync(kFull, old, 0);
        finish = old == nch - 1;
        if (finish) {
          __threadfence();
          const uint32_t first = ch.w - ((ch.z >> 10) & 0x1FFFFFu);
          C tot = (C)0;
          for (uint32_t c = lane; c < nch; c += 32) tot += ldcg(part + first + c);
          // lane order then a fixed shuffle tree: the same sum whichever warp finishes
          sum = warp_sum(tot);
          if (lane == 0) a.chunk_done[v] = 0;
        }
      }
      if (finish) {
        int exp_now = 0;
        if (lane == 0) {
          B dr = finish_at(v, sum, rold, ad);
          my_v++;
          my_e += deg;
          exp_now = expand && dr > a.ftol && first_expansion_pre(a.xbits, v, xw);
        }
        if constexpr (DF) {
          if (expand) queue_expansion(a, lane == 0 && exp_now, v, lane, wb);
        }
        if constexpr (CONT) record_expansion(a, lane == 0 && exp_now, v, lane, slot);
      }
    }

  io.my_max = my_max;
  io.dacc = dacc;
  *io.wb = wb;
  io.my_v = my_v;
  io.my_e = my_e;
  io.my_xv = my_xv;
  io.my_xe = my_xe;
  io.my_app = my_app;
}


// DF: compiled for Dynamic Frontier calls (marking and frontier expansion); Static and
// Naive-dynamic use the instance without them, which needs fewer registers.
// Dynamic Traversal (Section 3.3.2): breadth-first search from the seeds phase 0 marked (the
// sources, via their self-loops and new out-rows, and the deleted targets; together they reach
// exactly what the sources reach in G^{t-1} or G^t). Round r expands the vertices that joined
// in round r - 1; slot r's tails and hub queue keep rounds apart. When the search closes every
// stamp is reset to iteration 0. A search deeper than the round limit reports `all`: every
// vertex is then taken as affected.
struct DtOut {
  uint32_t cnt[3];
  uint32_t app, xv, xe, epoch;
  bool ok, all;
};
template <bool F32>
__device__ __noinline__ DtOut dt_search(const RankArgs<F32> &a, uint32_t epoch, uint32_t c0, uint32_t c1,
                                        uint32_t c2, WarpBuf *wbp) {
  __shared__ uint32_t s_err;
  const uint32_t tid = threadIdx.x, lane = tid & 31;
  const uint32_t nthreads = gridDim.x * kRankBlock;
  const uint32_t gtid = blockIdx.x * kRankBlock + tid;
  const uint32_t nwarps = nthreads >> 5, gwarp = gtid >> 5;
  RankCtl *ctl = a.ctl;
  DtOut o{{c0, c1, c2}, 0u, 0u, 0u, epoch, false, false};
  WarpBuf wb = *wbp;
  wb.dense = false;
  const uint32_t *lists[3] = {a.list0, a.list1, a.list2};
  uint32_t done[3] = {0u, 0u, 0u};
  uint32_t r = 1;
  for (; r <= (uint32_t)kMaxIterLimit; r++) {
#pragma unroll
    for (int bb = 0; bb < 3; bb++) {
      for (uint32_t k0 = done[bb] + gwarp * 32; k0 < o.cnt[bb]; k0 += nwarps * 32) {
        const bool p = k0 + lane < o.cnt[bb];
        const uint32_t x = p ? ldcg(lists[bb] + k0 + lane) : 0u;
        const ExpandOut e = expand_lanes(a, p ? 1 : 0, x, r, o.cnt[0], o.cnt[1], o.cnt[2], &wb);
        o.app += e.app;
        o.xv += e.xv;
        o.xe += e.xe;
      }
    }
    flush_marks(a, r, o.cnt, lane, wb);
    if (!grid_sync(ctl, o.epoch, &s_err)) return o;
    if (__ldcg(&ctl->hubq[r]) != 0) {
      o.app += hub_pass(a, r, o.cnt, lane, gwarp, nwarps, wb);
      flush_marks(a, r, o.cnt, lane, wb);
      if (!grid_sync(ctl, o.epoch, &s_err)) return o;
    }
    uint32_t added = 0;
#pragma unroll
    for (int bb = 0; bb < 3; bb++) {
      const uint32_t t = ldcg(&ctl->tail[r][bb]);
      done[bb] = o.cnt[bb];
      o.cnt[bb] += t;
      added += t;
    }
    if (added == 0) break;
  }
  if (r > (uint32_t)kMaxIterLimit) {
    o.all = true;
  } else {
#pragma unroll
    for (int bb = 0; bb < 3; bb++)
      for (uint32_t k = gtid; k < o.cnt[bb]; k += nthreads) a.stamp[ldcg(lists[bb] + k)] = 0;
    if (!grid_sync(ctl, o.epoch, &s_err)) return o;
  }
  *wbp = wb;
  o.ok = true;
  return o;
}

// SPLIT: the marking launch of a split call (single graph, self-loop mode), which hands the
// call to the per-iteration launches before its first dense iteration and before any
// iteration over every vertex; its instance carries no dense or full sweep code.
template <bool F32, bool DF, bool SPLIT = false>
__global__ void __launch_bounds__(kRankBlock, PRDF_RANK_MIN_BLOCKS) k_rank(const RankArgs<F32> a) {
  using S = Store<F32>;
  using R = typename S::R;
  using C = typename S::C;
  using B = typename Num<F32>::B;
  __shared__ uint32_t s_idx, s_err;
  __shared__ C s_part[kWarps];
  __shared__ unsigned long long s_key[kWarps];
  __shared__ double s_ds[kWarps], s_dc[kWarps];
  __shared__ int s_expand;
  __shared__ uint32_t s_mbuf[kWarps][4 * kMarkBuf];

  const uint32_t tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  const uint32_t nblk = gridDim.x;
  const uint32_t nthreads = nblk * kRankBlock;
  const uint32_t gtid = blockIdx.x * kRankBlock + tid;
  const uint32_t nwarps = nthreads >> 5, gwarp = gtid >> 5;
  RankCtl *ctl = a.ctl;
  uint32_t epoch = 0;
  constexpr bool df = DF;
  // per-component state (batched form), identical in every block; a split call's marking
  // launch serves one graph in self-loop mode (no components, no teleport)
  const bool multi = !SPLIT && a.ncomp > 1;
  const bool tele = !SPLIT && a.teleport;
  const uint32_t nc = a.ncomp;
  extern __shared__ unsigned long long dsm[];
  unsigned long long *s_kmax = dsm;                         // block max key / counter per component
  R *s_base = reinterpret_cast<R *>(dsm + nc);              // (1 - alpha) / n_c
  uint16_t *s_iters = reinterpret_cast<uint16_t *>(dsm + 2 * nc);
  uint8_t *s_active = reinterpret_cast<uint8_t *>(s_iters + nc);
  for (uint32_t c = tid; c < nc; c += kRankBlock) {
    s_kmax[c] = 0;
    s_base[c] = multi ? a.comp_base[c] : a.base;
    s_iters[c] = 0;
    s_active[c] = 1;
  }
  auto live = [&](uint32_t v) -> bool { return !multi || s_active[__ldg(a.comp + v)]; };
#define pol_cols l2_evict_first()
#define pol_c l2_evict_last()
  uint32_t my_v = 0, my_e = 0, my_xv = 0, my_xe = 0, my_app = 0;  // per-thread, folded at the end

  // dead-end mass: per-block partials (double-buffered by parity) and their grid total
  Mass<F32> dacc;
  auto block_dead_partial = [&](int parity) {
    if constexpr (F32) {
      double s = dacc.n.s, c = dacc.n.c;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        double os = __shfl_xor_sync(kFull, s, o), oc = __shfl_xor_sync(kFull, c, o);
        Neu t;
        t.s = s;
        t.c = c;
        t.merge(os, oc);
        s = t.s;
        c = t.c;
      }
      if (lane == 0) {
        s_ds[wib] = s;
        s_dc[wib] = c;
      }
      __syncthreads();
      if (tid == 0) {
        Neu t;
        for (int w = 0; w < kWarps; w++) t.merge(s_ds[w], s_dc[w]);
        a.dpart[parity * nblk + blockIdx.x] = DeadPart{t.s, t.c};
      }
    } else {
      long long s = warp_sum(dacc.s);
      if (lane == 0) s_ds[wib] = __longlong_as_double(s);
      __syncthreads();
      if (tid == 0) {
        long long t = 0;
        for (int w = 0; w < kWarps; w++) t += __double_as_longlong(s_ds[w]);
        a.dpart[parity * nblk + blockIdx.x] = DeadPart{__longlong_as_double(t), 0.0};
      }
    }
    dacc = Mass<F32>();
  };
  // the grid total, as a rank-representation value (exact sum in 64-bit mode)
  auto grid_dead_total = [&](int parity, double *as_double) -> long long {
    if constexpr (F32) {
      Neu t;
      for (uint32_t k = 0; k < nblk; k++) {
        const double *p = &a.dpart[parity * nblk + k].s;
        t.merge(__ldcg(p), __ldcg(p + 1));
      }
      *as_double = t.s + t.c;
      return 0;
    } else {
      long long t = 0;
      for (uint32_t k = 0; k < nblk; k++)
        t += __double_as_longlong(__ldcg(&a.dpart[parity * nblk + k].s));
      *as_double = 0.0;
      return t;
    }
  };
  // alpha D / n in the rank representation
  auto tele_of = [&](long long Dn, double Dd) -> R {
    if constexpr (F32) return (float)(a.tele_d * Dd);
    else return S::contrib(Dn, a.tele_frac);
  };

  if (blockIdx.x == 0 && tid == 0) ctl->t_ns[0] = globaltimer_ns();

  // ---------------------------------------------------------------- phase 0
  if (a.mode == kModeStatic) {
    for (uint32_t v = gtid; v < a.n; v += nthreads) {
      const R r = multi ? a.comp_init[__ldg(a.comp + v)] : a.init;
      C c = S::contrib(r, __ldg(a.adeg + v));
      a.R0[v] = r;
      a.R1[v] = r;
      a.C0[v] = c;
      a.C1[v] = c;
    }
    if (tele)
      for (uint32_t k = gtid; k < a.n_dead; k += nthreads) dacc.add(a.init);
  } else if (tele) {
    for (uint32_t k = gtid; k < a.n_dead; k += nthreads) dacc.add(ldcg(a.R0 + __ldg(a.dead + k)));
  }
  const uint32_t zero_cnt[3] = {0, 0, 0};
  WarpBuf wb{s_mbuf[wib], {0u, 0u, 0u, 0u}, false, 0u};
  // expansion-list entries already scanned; read before any barrier of this launch, since
  // the sweeps append to the list once the first barrier is passed
  uint32_t xdone = 0;
  if (df && !a.start_full) {
    // sources: mark G^t.out(u), 32 sources per warp round (short rows by their own lanes,
    // medium rows flattened over the warp, long rows by the whole grid)
    for (uint32_t k0 = gwarp * 32; k0 < a.n_pend_src; k0 += nwarps * 32) {
      const bool p = k0 + lane < a.n_pend_src;
      const uint32_t u = p ? __ldg(a.pend_src + k0 + lane) : 0u;
      const ExpandOut o = expand_lanes(a, p ? 1 : 0, u, 0u, 0u, 0u, 0u, &wb);
      my_app += o.app;
      my_xv += o.xv;
      my_xe += o.xe;
    }
    // deleted targets, 32 per warp round
    for (uint32_t k0 = gwarp * 32; k0 < a.n_pend_tgt; k0 += nwarps * 32) {
      uint32_t cnt_left = min(32u, a.n_pend_tgt - k0);
      my_app += warp_mark_range(a, a.pend_tgt + k0, cnt_left, 0, 32, 0, zero_cnt, lane, wb);
    }
  }
  flush_marks(a, 0u, zero_cnt, lane, wb);
  if (tele) block_dead_partial(0);
  if (!grid_sync(ctl, epoch, &s_err)) return;
  if (df && __ldcg(&ctl->hubq[0]) != 0) {
    my_app += hub_pass(a, 0, zero_cnt, lane, gwarp, nwarps, wb);
    flush_marks(a, 0u, zero_cnt, lane, wb);
    if (!grid_sync(ctl, epoch, &s_err)) return;
  }
  if (blockIdx.x == 0 && tid == 0) ctl->t_ns[1] = globaltimer_ns();

  uint32_t cnt[3];
#pragma unroll
  for (int bb = 0; bb < 3; bb++) cnt[bb] = df && !a.start_full ? ldcg(&ctl->tail[0][bb]) : 0u;
  // counters of a launch that stops early and leaves the iterations to other launches
  auto fold_counters = [&]() {
    const unsigned long long xv = warp_sum((unsigned long long)my_xv), xe = warp_sum((unsigned long long)my_xe),
                             ap = warp_sum((unsigned long long)my_app);
    if (lane == 0) {
      if (xv) atomicAdd(&ctl->expv, xv);
      if (xe) atomicAdd(&ctl->expe, xe);
      if (ap) atomicAdd(&ctl->appended, ap);
    }
  };
  // Dynamic Traversal: every vertex reachable from the seeds phase 0 marked joins iteration 0
  // and nothing is marked afterwards
  const bool dt = df && a.mode == kModeDT;
  bool dt_all = false;
  if (dt && !a.start_full) {
    const DtOut o = dt_search(a, epoch, cnt[0], cnt[1], cnt[2], &wb);
    if (!o.ok) return;
    epoch = o.epoch;
#pragma unroll
    for (int bb = 0; bb < 3; bb++) cnt[bb] = o.cnt[bb];
    my_app += o.app;
    my_xv += o.xv;
    my_xe += o.xe;
    dt_all = o.all;
    if (dt_all && blockIdx.x == 0 && tid == 0) ctl->full_from = 1u;
    if (blockIdx.x == 0 && tid == 0) ctl->t_ns[1] = globaltimer_ns();
    if (dt_all && a.split) {
      // every vertex is affected, so the iterations are those of Naive-dynamic: the search's
      // marks are cleared and the host runs the iterations in the full-sweep instance, which
      // carries none of the marking code
      const uint32_t *lists[3] = {a.list0, a.list1, a.list2};
#pragma unroll
      for (int bb = 0; bb < 3; bb++)
        for (uint32_t k = gtid; k < cnt[bb]; k += nthreads) {
          const uint32_t v = ldcg(lists[bb] + k);
          a.bitmap[v >> 5] = 0u;
          a.xbits[v >> 5] = 0u;
          a.stamp[v] = kNoStamp;
        }
      fold_counters();
      if (blockIdx.x == 0 && tid == 0) ctl->status = kStatusFull;
      return;
    }
    if (a.split) {
      // the set is fixed: every iteration runs in the per-iteration launches
      fold_counters();
      if (blockIdx.x == 0 && tid == 0) {
#pragma unroll
        for (int bb = 0; bb < 3; bb++) ctl->save_cnt[bb] = cnt[bb];
        ctl->next_it = 0;
        ctl->status = kStatusDense;
      }
      return;
    }
  }
  long long Dn = 0;
  double Dd = 0.0;
  if (tele) Dn = grid_dead_total(0, &Dd);
  R tele_prev = tele ? tele_of(a.D_ref_n, a.D_ref_d) : (R)0;
  bool ever_full = !df || a.start_full || dt_all;
  uint32_t iters = 0;
  bool converged = false;
  unsigned long long last_key = 0;
  const uint32_t dense_at = a.n / a.dense_div;
  uint32_t cmp_total = 0xFFFFFFFFu;  // affected count at the last compaction (none yet)
  uint32_t prev_total = 0xFFFFFFFFu; // affected count at the start of the previous iteration
  uint32_t cmp_n[3] = {0, 0, 0};
  uint32_t deact = 0, cmp_deact = 0;  // iterations in which some graph stopped (batched form)
  bool handed_off = false;

  // ------------------------------------------------------------- iterations
  for (int it = 0; it < a.max_iter; it++) {
    Iter<F32> I;
    I.tele = tele ? tele_of(Dn, Dd) : (R)0;
    if (df && tele && !ever_full && Num<F32>::delta(I.tele, tele_prev) > a.ftol) {
      // the teleport term of every vertex moved by more than tau_f: all of V is affected
      ever_full = true;
      if (blockIdx.x == 0 && tid == 0) ctl->full_from = (uint32_t)it + 1;
    }
    tele_prev = I.tele;
    I.full = ever_full;
    const int par = it & 1;
    const R *Rin = par ? a.R1 : a.R0;
    const C *Cin = par ? a.C1 : a.C0;
    R *Rout = par ? a.R0 : a.R1;
    C *Cout = par ? a.C0 : a.C1;
    // dense: once the affected lists are large, iterate over the sweep items of the affected
    // vertices (compacted from all items whenever the affected set grew), in tier order
    const bool dense = !I.full && (cnt[0] + cnt[1] + cnt[2] > dense_at);
    // dense iterations sweep the compacted items of the affected vertices, compacted again
    // when the set changed; a set that is large (over n / 4) and still growing by more than
    // 1/16 per iteration is instead swept through all items, skipping vertices stamped later
    // than it
    const uint32_t total_now = cnt[0] + cnt[1] + cnt[2];
    const bool scan_all = dense && total_now != cmp_total && total_now > a.n / 4 &&
                          (prev_total == 0xFFFFFFFFu || total_now - prev_total > total_now / 16);
    prev_total = total_now;
    // split calls: once the affected set is dense, the iterations continue in the
    // per-iteration launches (which grow the set by pulling or pushing); this launch stops
    // before the iteration, whose marks are in place
    if (df && a.split && dense) {
      if (blockIdx.x == 0 && tid == 0) {
#pragma unroll
        for (int bb = 0; bb < 3; bb++) ctl->save_cnt[bb] = cnt[bb];
        ctl->next_it = (uint32_t)it;
        ctl->status = kStatusDense;
      }
      handed_off = true;
      break;
    }
    const bool expand = df && !dt && !I.full;
    // split calls: a sparse iteration over a set whose out-rows would likely make the next
    // set dense (defer_at, from the average degree) pushes nothing; it records each
    // vertex's change flag (and marks the first expansions as done), and the next
    // iteration, the first of the per-iteration launches, pulls its marks from them
    // (pushing that many out-rows costs more than one pull over every item)
    const bool defer = expand && a.split && !dense && total_now > a.defer_at;
    const uint32_t slot = (uint32_t)it + 1;
    B my_max = 0;
    if (blockIdx.x == 0 && tid == 0) {
      ctl->it_aff[it] = I.full ? a.n : cnt[0] + cnt[1] + cnt[2];
      ctl->it_kind[it] =
          I.full ? 3 : (scan_all ? 4 : (dense ? (cnt[0] + cnt[1] + cnt[2] != cmp_total ? 2 : 1) : 0));
    }

    wb.dense = dense;
    wb.slot = slot;

    auto expand_if = [&](int push, uint32_t v) {
      if (__any_sync(kFull, push)) {
        const ExpandOut o = expand_lanes(a, push, v, slot, cnt[0], cnt[1], cnt[2], &wb);
        my_app += o.app;
        my_xv += o.xv;
        my_xe += o.xe;
      }
    };

    // rank of v from its in-sum; notes |change| in the (per-component) L-inf max
    auto finish_at = [&](uint32_t v, C sum, R rold, typename S::A ad) -> B {
      const uint32_t c = multi ? (uint32_t)__ldg(a.comp + v) : 0u;
      const B dr = finish_vertex(a, Rout, Cout, v, sum, rold, ad, I, dacc, pol_c, multi ? s_base[c] : a.base);
      if (multi) atomicMax(&s_kmax[c], Num<F32>::key(dr));
      else my_max = dr > my_max ? dr : my_max;
      return dr;
    };
    // sparse iterations: whether v's out-row is marked now; a deferred iteration records
    // the change flag instead (the out-row is then marked by the next iteration's pull)
    auto sparse_push = [&](uint32_t v, B dr) -> int {
      if (!expand) return 0;
      const bool big = dr > a.ftol;
      if (defer) {
        a.emap[(size_t)(it & 1) * a.n + v] = big ? 1 : 0;
        if (big) first_expansion(a.xbits, v);
        return 0;
      }
      return big && first_expansion(a.xbits, v);
    };

    if (!SPLIT && (I.full || dense)) {
      const uint32_t off1 = a.it_c0, off2 = a.it_c0 + a.it_c1;
      const uint4 *T = a.items;
      uint32_t n0 = a.it_c0, n1 = a.it_c1, n2 = a.it_c2;
      auto take = [&](uint32_t v) -> bool {
        return live(v) && (!scan_all || ldcg(a.stamp + v) <= (uint16_t)it);
      };
      if (dense && !scan_all) {
        const uint32_t total = cnt[0] + cnt[1] + cnt[2];
        if (total != cmp_total || deact != cmp_deact) {
          // keep the items of vertices stamped <= it; warp-aggregated appends keep runs of
          // up to 32 items in tier order
          const uint32_t segs[3][2] = {{0u, a.it_c0}, {off1, a.it_c1}, {off2, a.it_c2}};
#pragma unroll
          for (int t = 0; t < 3; t++) {
            const uint32_t base = segs[t][0], cntt = segs[t][1];
            for (uint32_t b0 = gwarp * 32; b0 < cntt; b0 += nwarps * 32) {
              const uint32_t i = b0 + lane;
              uint4 item = make_uint4(0, 0, 0, 0);
              bool keep = false;
              if (i < cntt) {
                item = __ldg(a.items + base + i);
                keep = ldcg(a.stamp + item.x) <= (uint16_t)it && live(item.x);
              }
              const uint32_t mask = __ballot_sync(kFull, keep);
              if (mask) {
                const uint32_t leader = __ffs(mask) - 1;
                uint32_t at = 0;
                if (lane == leader) at = atomicAdd(&ctl->cmp[slot][t], (uint32_t)__popc(mask));
                at = __shfl_sync(kFull, at, leader);
                if (keep) a.items_cmp[base + at + __popc(mask & lanemask_lt())] = item;
              }
            }
          }
          if (!grid_sync(ctl, epoch, &s_err)) return;
#pragma unroll
          for (int t = 0; t < 3; t++) cmp_n[t] = ldcg(&ctl->cmp[slot][t]);
          cmp_total = total;
          cmp_deact = deact;
        }
        T = a.items_cmp;
        n0 = cmp_n[0];
        n1 = cmp_n[1];
        n2 = cmp_n[2];
      }

      SweepIo<F32> io;
      io.Rin = Rin;
      io.Cin = Cin;
      io.Rout = Rout;
      io.Cout = Cout;
      io.T = T;
      io.n0 = n0;
      io.n1 = n1;
      io.n2 = n2;
      io.off1 = off1;
      io.off2 = off2;
      io.it = (uint32_t)it;
      io.slot = slot;
      io.cnt[0] = cnt[0];
      io.cnt[1] = cnt[1];
      io.cnt[2] = cnt[2];
      io.scan_all = scan_all;
      io.expand = expand;
      io.I = I;
      io.s_base = s_base;
      io.s_kmax = s_kmax;
      io.s_active = s_active;
      io.wb = &wb;
      io.dacc = dacc;
      io.my_max = my_max;
      sweep_tiers<F32, DF ? 1 : 0>(a, io);
      my_max = io.my_max;
      dacc = io.dacc;
      my_v += io.my_v;
      my_e += io.my_e;
      my_xv += io.my_xv;
      my_xe += io.my_xe;
      my_app += io.my_app;
    } else {
      // sparse: thread bin, one thread per vertex, 32 consecutive list entries per warp
      for (uint32_t b0 = gwarp * 32; b0 < cnt[0]; b0 += nwarps * 32) {
        const uint32_t i = b0 + lane;
        int push = 0;
        uint32_t v = 0;
        if (i < cnt[0] && live(ldcg(a.list0 + i))) {
          v = ldcg(a.list0 + i);
          const R rold = ldcg(Rin + v);
          const typename S::A ad = __ldg(a.adeg + v);
          const uint2 d = __ldg(&a.in_rd[v]);
          C sum = row_sum_thread(Cin, a.in_col + d.x, d.y, pol_cols, pol_c);
          B dr = finish_at(v, sum, rold, ad);
          my_v++;
          my_e += d.y;
          push = sparse_push(v, dr);
        }
        if (expand) expand_if(push, v);
      }

      // sparse: warp bin, one warp per vertex
      for (uint32_t i = gwarp; i < cnt[1]; i += nwarps) {
        const uint32_t v = ldcg(a.list1 + i);
        if (!live(v)) continue;
        const uint2 d = __ldg(&a.in_rd[v]);
        const uint32_t *cols = a.in_col + d.x;
        C sum = (C)0;
        for (uint32_t j = lane * 4; j < d.y; j += 128) {
          uint4 q = ld_cols(cols + j, pol_cols);
          sum += gather4(Cin, q, min(4u, d.y - j), pol_c);
        }
        sum = warp_sum(sum);
        int exp_now = 0;
        if (lane == 0) {
          B dr = finish_at(v, sum, ldcg(Rin + v), __ldg(a.adeg + v));
          my_v++;
          my_e += d.y;
          exp_now = sparse_push(v, dr);
        }
        exp_now = __shfl_sync(kFull, exp_now, 0);
        if (exp_now) {
          const ExpandOut o = expand_one(a, v, slot, cnt[0], cnt[1], cnt[2], &wb);
          my_app += o.app;
          my_xv += o.xv;
          my_xe += o.xe;
        }
      }

      // sparse: block bin, one block per vertex, taken dynamically
      for (;;) {
        if (tid == 0) s_idx = atomicAdd(&ctl->blk_next[it], 1u);
        __syncthreads();
        const uint32_t idx = s_idx;
        __syncthreads();
        if (idx >= cnt[2]) break;
        const uint32_t v = ldcg(a.list2 + idx);
        if (!live(v)) continue;
        const uint2 d = __ldg(&a.in_rd[v]);
        const uint32_t *cols = a.in_col + d.x;
        C sum = (C)0;
        for (uint32_t j0 = tid * 4; j0 < d.y; j0 += kRankBlock * 16) {
          uint4 q[4];
#pragma unroll
          for (int r = 0; r < 4; r++) {
            const uint32_t j = j0 + r * kRankBlock * 4;
            if (j < d.y) q[r] = ld_cols(cols + j, pol_cols);
          }
#pragma unroll
          for (int r = 0; r < 4; r++) {
            const uint32_t j = j0 + r * kRankBlock * 4;
            if (j < d.y) sum += gather4(Cin, q[r], min(4u, d.y - j), pol_c);
          }
        }
        sum = warp_sum(sum);
        if (lane == 0) s_part[wib] = sum;
        __syncthreads();
        if (tid == 0) {
          C tot = (C)0;
          for (int w = 0; w < kWarps; w++) tot += s_part[w];
          B dr = finish_at(v, tot, ldcg(Rin + v), __ldg(a.adeg + v));
          my_v++;
          my_e += d.y;
          s_expand = sparse_push(v, dr);
        }
        __syncthreads();
        if (s_expand) {
          const uint2 od = __ldg(&a.out_rd[v]);
          if (od.y <= kInlineOut) {
            my_app += warp_mark_range(a, a.out_col + od.x, od.y, wib * 32, kRankBlock, slot, cnt, lane, wb);
          } else if (wib == 0) {
            my_app += expand_vertex(a, v, od, slot, cnt, lane, wb);
          }
          if (tid == 0) {
            my_xv++;
            my_xe += od.y;
          }
        }
      }
    }

    if (expand) flush_marks(a, slot, cnt, lane, wb);

    // block reductions: L-inf (and dead-end mass) of this iteration
    if (multi) {
      __syncthreads();
      unsigned long long *cur = a.dRc + (uint64_t)(it % 3) * nc;
      unsigned long long *nxt = a.dRc + (uint64_t)((it + 1) % 3) * nc;
      for (uint32_t c = tid; c < nc; c += kRankBlock) {
        if (s_kmax[c]) atomicMax(cur + c, s_kmax[c]);
        s_kmax[c] = 0;
        if (blockIdx.x == 0) nxt[c] = 0;  // last read two iterations ago, before the previous barrier
      }
    } else {
      unsigned long long m = Num<F32>::key(my_max);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
      if (lane == 0) s_key[wib] = m;
      __syncthreads();
      if (tid == 0) {
        unsigned long long bm = 0;
        for (int w = 0; w < kWarps; w++) bm = max(bm, s_key[w]);
        if (bm) atomicMax(&ctl->dR_bits[it], bm);
      }
    }
    if (tele) block_dead_partial((it + 1) & 1);
    if (!grid_sync(ctl, epoch, &s_err)) return;
    if (expand) {
      // out-rows of the vertices this iteration's sweep queued, 32 per warp round, one
      // vertex per lane; rows longer than 128 go to the hub queue
      const uint32_t xend = xdone + ldcg(&ctl->xit[slot]);
      if (xend > xdone) {
        for (uint32_t k0 = xdone + gwarp * 32; k0 < xend; k0 += nwarps * 32) {
          const bool p = k0 + lane < xend;
          const uint32_t x = p ? ldcg(a.xlist + k0 + lane) : 0u;
          const ExpandOut o = expand_lanes(a, p ? 1 : 0, x, slot, cnt[0], cnt[1], cnt[2], &wb);
          my_app += o.app;
          my_xv += o.xv;
          my_xe += o.xe;
        }
        xdone = xend;
        flush_marks(a, slot, cnt, lane, wb);
        if (!grid_sync(ctl, epoch, &s_err)) return;
      }
    }
    if (expand && __ldcg(&ctl->hubq[slot]) != 0) {
      my_app += hub_pass(a, slot, cnt, lane, gwarp, nwarps, wb);
      flush_marks(a, slot, cnt, lane, wb);
      if (!grid_sync(ctl, epoch, &s_err)) return;
    }

    unsigned long long dR = __ldcg(&ctl->dR_bits[it]);
    int any_active = 1;
    if (multi) {
      // every block applies the same per-component convergence decisions
      const unsigned long long *cur = a.dRc + (uint64_t)(it % 3) * nc;
      int act = 0, stopped = 0;
      unsigned long long mx = 0;
      for (uint32_t c = tid; c < nc; c += kRankBlock) {
        if (!s_active[c]) continue;
        const unsigned long long k = __ldcg(cur + c);
        mx = k > mx ? k : mx;
        s_iters[c] = (uint16_t)(it + 1);
        const bool done = k <= a.tol_key;
        if (done || it + 1 == a.max_iter) {
          s_active[c] = 0;
          stopped = 1;
          if (blockIdx.x == 0) {
            a.comp_out[4 * c + 0] = (uint32_t)it + 1;
            a.comp_out[4 * c + 1] = done ? 1u : 0u;
            a.comp_last[c] = k;
          }
        } else {
          act = 1;
        }
      }
      any_active = __syncthreads_or(act);
      if (__syncthreads_or(stopped)) deact++;
      if (blockIdx.x == 0) {
        // combined L-inf of this iteration for the call's stats
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
        if (lane == 0 && mx) atomicMax(&ctl->dR_bits[it], mx);
      }
      dR = any_active ? a.tol_key + 1 : 0;  // stop when no component is still iterating
    }
    if (expand) {
#pragma unroll
      for (int bb = 0; bb < 3; bb++) cnt[bb] += ldcg(&ctl->tail[slot][bb]);
    }
    if (tele) {
      double pd = 0.0;
      long long pn = grid_dead_total((it + 1) & 1, &pd);
      if (I.full) {
        Dn = pn;
        Dd = pd;
      } else {
        Dn += pn;
        Dd += pd;
      }
    }
    iters = (uint32_t)it + 1;
    last_key = dR;
    if (blockIdx.x == 0 && tid == 0) ctl->t_ns[it + 2] = globaltimer_ns();
    if (defer) {
      // tier-2 rows pull before the handoff (the first per-iteration sweep pulls tier-0/1
      // rows itself).  If this was the last iteration (converged or max_iter), the launches
      // that follow only make its marks, which belong to the affected set (Algorithm 1
      // marks in every iteration, the last included)
      const bool last = dR <= a.tol_key || it + 1 >= a.max_iter;
      my_app += pull_tier2(a, slot, cnt[0], a.it_c2, a.it_c0 + a.it_c1);
      if (!grid_sync(ctl, epoch, &s_err)) return;
      if (blockIdx.x == 0 && tid == 0) {
#pragma unroll
        for (int bb = 0; bb < 3; bb++) ctl->save_cnt[bb] = cnt[bb] + (bb == 0 ? ldcg(&ctl->tail[slot][0]) : 0u);
        ctl->next_it = slot;
        ctl->pull_check = 1;
        ctl->fin_only = last ? 1u : 0u;
        ctl->iterations = slot;
        ctl->converged = dR <= a.tol_key ? 1u : 0u;
        ctl->last_key = dR;
        ctl->status = kStatusDense;
      }
      handed_off = true;
      break;
    }
    if (dR <= a.tol_key) {
      converged = true;
      break;
    }
  }

  // -------------------------------------------------------------- writeback
  // the final values of a vertex are in parity (its component's iterations) & 1; copy them
  // to the other parity so both hold the current ranks
  auto copy_final = [&](uint32_t v) {
    const uint32_t k = multi ? s_iters[__ldg(a.comp + v)] : iters;
    const bool fp = k & 1;
    const R *Rf = fp ? a.R1 : a.R0;
    const C *Cf = fp ? a.C1 : a.C0;
    R *Ro = fp ? a.R0 : a.R1;
    C *Co = fp ? a.C0 : a.C1;
    Ro[v] = ldcg(Rf + v);
    Co[v] = ldcg(Cf + v);
  };
  __syncthreads();
  if (ever_full)
    for (uint32_t v = gtid; v < a.n; v += nthreads) copy_final(v);
  if (df && !handed_off) {
    const uint32_t *lists[3] = {a.list0, a.list1, a.list2};
    for (int bb = 0; bb < 3; bb++) {
      for (uint32_t k = gtid; k < cnt[bb]; k += nthreads) {
        const uint32_t v = ldcg(lists[bb] + k);
        if (!ever_full) copy_final(v);
        if (multi) atomicAdd(&s_kmax[__ldg(a.comp + v)], 1ull);
        a.bitmap[v >> 5] = 0u;
        a.xbits[v >> 5] = 0u;
        a.stamp[v] = kNoStamp;
        if (a.emap) {
          a.emap[v] = 0;
          a.emap[a.n + v] = 0;
        }
      }
    }
    if (multi) {
      __syncthreads();
      for (uint32_t c = tid; c < nc; c += kRankBlock)
        if (s_kmax[c]) atomicAdd(&a.comp_out[4 * c + 2], (uint32_t)s_kmax[c]);
    }
  }
  // counters
  {
    unsigned long long vals[5] = {my_v, my_e, my_xv, my_xe, my_app};  // widened before the warp sums
    unsigned long long *dst[5] = {&ctl->vproc, &ctl->eproc, &ctl->expv, &ctl->expe, &ctl->appended};
#pragma unroll
    for (int k = 0; k < 5; k++) {
      unsigned long long x = warp_sum(vals[k]);
      if (lane == 0 && x) atomicAdd(dst[k], x);
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
    for (int bb = 0; bb < 3; bb++) ctl->final_cnt[bb] = cnt[bb];
    if (!handed_off) {
      ctl->iterations = iters;
      ctl->converged = converged ? 1u : 0u;
      ctl->last_key = last_key;
      ctl->D_final = Dd;
      ctl->D_final_n = Dn;
      ctl->status = kStatusDone;
    }
  }
}

#undef pol_cols
#undef pol_c

// ------------------------------------------------------------------ host side ---

#define CK(call)                                            \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(g, e_, #call);  \
  } while (0)

static constexpr double kOne62 = 4611686018427387904.0;  // 2^62

// Dynamic shared memory of k_rank: per-component max key, base, iteration count, active flag.
static size_t rank_smem(uint32_t ncomp) { return ((size_t)ncomp * 19 + 15) & ~(size_t)15; }

template <bool F32>
static cudaError_t grid_blocks(int sm_count, size_t smem, int *blocks) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rank<F32, false>, kRankBlock, smem);
  if (e != cudaSuccess) return e;
  int per_sm_df = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_df, k_rank<F32, true>, kRankBlock, smem);
  if (e != cudaSuccess) return e;
  per_sm = std::min(per_sm, per_sm_df);
  per_sm = std::max(1, std::min(per_sm, 4));
  *blocks = per_sm * sm_count;
  return cudaSuccess;
}

pr_status rank_setup(Graph *g) {
  int blocks = 0;
  const size_t smem = rank_smem(g->ncomp);
  CK(g->f32 ? grid_blocks<true>(g->sm_count, smem, &blocks) : grid_blocks<false>(g->sm_count, smem, &blocks));
  g->rank_grid = blocks;
  g->rank_grid_max = blocks;
  CK(cudaMalloc((void **)&g->ctl, sizeof(RankCtl)));
  CK(cudaMallocHost((void **)&g->ctl_h, sizeof(RankCtl)));
  CK(cudaMalloc((void **)&g->dpart, sizeof(DeadPart) * 2 * (size_t)blocks));
  CK(cudaEventCreate(&g->ev0));
  CK(cudaEventCreate(&g->ev1));
  return sweep_setup(g);
}

// The full-sweep instance in Naive-dynamic mode on the arguments of a marking call whose
// affected set is all of V (nothing to mark, every vertex iterated from the current ranks).
template <bool F32>
static cudaError_t launch_full_sweep(Graph *g, const RankArgs<F32> &a) {
  RankArgs<F32> b = a;
  b.mode = (int)kModeNaive;
  b.start_full = 0;
  b.split = 0;
  void *args[] = {(void *)&b};
  cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_rank<F32, false>, dim3(g->rank_grid), dim3(kRankBlock),
                                              args, rank_smem(g->ncomp), g->st);
  if (e == cudaSuccess) count_launch();
  return e;
}

template <bool F32>
static pr_status launch(Graph *g, RankMode mode, bool start_full) {
  using S = Store<F32>;
  RankArgs<F32> a{};
  const double n = (double)g->n, alpha = g->p.alpha;
  a.n = g->n;
  a.in_rd = g->in.rd;
  a.in_col = g->in.col;
  a.out_rd = g->out.rd;
  a.out_col = g->out.col;
  a.R0 = (typename S::R *)g->R[0];
  a.R1 = (typename S::R *)g->R[1];
  a.C0 = (typename S::C *)g->C[0];
  a.C1 = (typename S::C *)g->C[1];
  a.adeg = (const typename S::A *)g->adeg;
  a.bitmap = g->bitmap;
  a.xbits = g->xbits;
  a.stamp = g->stamp;
  a.list0 = g->list[0];
  a.list1 = g->list[1];
  a.list2 = g->list[2];
  a.items = g->items;
  a.items_cmp = g->items_cmp;
  a.it_c0 = g->item_cnt[0];
  a.it_c1 = g->item_cnt[1];
  a.it_c2 = g->item_cnt[2];
  a.partials = (typename S::C *)g->partials;
  a.chunk_done = g->chunk_done;
  a.hub_v = g->hub_v;
  a.hub_base = g->hub_base;
  a.pend_src = g->pend_src;
  a.n_pend_src = g->n_pend_src;
  a.pend_tgt = g->pend_tgt;
  a.n_pend_tgt = g->n_pend_tgt;
  a.dead = g->dead;
  a.n_dead = g->teleport ? g->n_dead : 0;
  a.dpart = g->dpart;
  if constexpr (F32) {
    a.base = (float)((1.0 - alpha) / n);
    a.init = (float)(1.0 / n);
    float ft = (float)g->p.frontier_tol;
    std::memcpy(&a.ftol, &ft, 4);
    double tl = g->p.tol;
    std::memcpy(&a.tol_key, &tl, 8);
    a.tele_d = alpha / n;
  } else {
    a.base = std::llrint((1.0 - alpha) / n * kOne62);
    a.init = std::llrint(1.0 / n * kOne62);
    a.ftol = (unsigned long long)std::floor(std::min(g->p.frontier_tol * kOne62, 9.0e18));
    a.tol_key = (unsigned long long)std::floor(std::min(g->p.tol * kOne62, 9.0e18));
    a.tele_frac = (unsigned long long)(alpha / n * 18446744073709551616.0);  // < 2^64 since alpha < 1
  }
  a.D_ref_n = g->D_ref_n;
  a.D_ref_d = g->D_ref;
  a.teleport = g->teleport ? 1 : 0;
  a.max_iter = g->p.max_iter;
  // asynchronous Dynamic Frontier (Section 4.2): one rank and one contribution vector, read
  // and written in place, so a vertex sees the ranks its in-neighbours already updated in the
  // same iteration; the marking instance runs unchanged on the aliased buffers
  const bool async = mode == kModeDFAsync;
  if (async) {
    a.R1 = a.R0;
    a.C1 = a.C0;
  }
  a.mode = (int)(async ? kModeDF : mode);
  a.start_full = start_full ? 1 : 0;
  a.bin_lo = (uint32_t)g->p.bin_lo;
  a.bin_hi = (uint32_t)g->p.bin_hi;
  a.gmax = g->group_max;
  a.chunk = g->chunk_len;
  a.ctl = g->ctl;
  a.ncomp = g->ncomp;
  a.comp = g->comp;
  a.comp_base = (const typename S::R *)g->comp_base;
  a.comp_init = (const typename S::R *)g->comp_init;
  a.dRc = g->dRc;
  a.comp_out = g->comp_out;
  a.comp_last = g->comp_last;
  a.dense_div = g->dense_div;
  a.xlist = g->xlist;
  a.emap = g->emap;
  a.item_pos = g->item_pos;
  const bool marking = mode == kModeDF || mode == kModeDT || async;
  const bool loops = sweep_eligible(g);
  a.split = marking && loops && g->split_df && !start_full;
  // expected marks of a set of k vertices: k * m / n; deferring to a pull pays once they
  // would make the next set dense (more than n / dense_div) several times over: a pull
  // reads the in-rows of every vertex not yet affected, so below that a push is cheaper
  // (4x measured best of 1/4x, 1x, 4x and 16x on R-MAT scale 22)
  a.defer_at = (uint32_t)std::min<double>((double)g->n, 4.0 * (double)g->n * (double)g->n /
                                                            ((double)g->dense_div * std::max<double>(1.0, (double)g->m)));
  void *args[] = {(void *)&a};
  auto copy_async_parity = [&]() -> pr_status {
    if (async) {  // the second parity takes the in-place result
      CK(cudaMemcpyAsync(g->R[1], g->R[0], sizeof(typename S::R) * (size_t)g->n, cudaMemcpyDeviceToDevice, g->st));
      CK(cudaMemcpyAsync(g->C[1], g->C[0], sizeof(typename S::C) * (size_t)g->n, cudaMemcpyDeviceToDevice, g->st));
    }
    return PR_OK;
  };
  if (loops && (!marking || start_full)) {
    // every vertex every iteration (Static; Naive-dynamic, also for a marking call whose
    // affected set is all of V): per-iteration launches in a device-side loop
    pr_status rc = sweep_full(g, mode == kModeStatic);
    if (rc != PR_OK) return rc;
    return copy_async_parity();
  }
  if (marking && start_full && !g->use_graph) {
    // every vertex is affected from iteration 0 and nothing is ever marked: Naive-dynamic
    CK(launch_full_sweep<F32>(g, a));
    return copy_async_parity();
  }
  const void *fn = marking ? (a.split && !g->use_graph ? (const void *)k_rank<F32, true, true> : (const void *)k_rank<F32, true>)
                           : (const void *)k_rank<F32, false>;
  if (!g->use_graph) {
    CK(cudaLaunchCooperativeKernel(fn, dim3(g->rank_grid), dim3(kRankBlock), args,
                                   rank_smem(g->ncomp), g->st));
    count_launch();
    if (a.split) {
      // the marking launch stops once the affected set is dense (or, for Dynamic
      // Traversal, after its search); the host reads the status it left and starts the
      // per-iteration loop, or the full sweeps if every vertex turned out affected
      CK(cudaMemcpyAsync(g->ctl_h, g->ctl, offsetof(RankCtl, final_cnt), cudaMemcpyDeviceToHost, g->st));
      CK(cudaStreamSynchronize(g->st));
      const RankCtl &h = *g->ctl_h;
      pr_status rc = PR_OK;
      if (!h.err && h.status == kStatusFull) rc = sweep_full(g, false);
      else if (!h.err && h.status == kStatusDense) rc = sweep_dense(g, mode, &a);
      if (rc != PR_OK) return rc;
    }
    return copy_async_parity();
  }
  // CUDA-graph launch: the control-block reset, the event records and the cooperative
  // kernel are captured once; later calls only replace the kernel's arguments and replay
  cudaKernelNodeParams kp{};
  kp.func = const_cast<void *>(fn);
  kp.gridDim = dim3(g->rank_grid);
  kp.blockDim = dim3(kRankBlock);
  kp.sharedMemBytes = (unsigned)rank_smem(g->ncomp);
  kp.kernelParams = args;
  if (g->cg_exec && (g->cg_f32 != F32 || g->cg_df != marking)) {
    cudaGraphExecDestroy(g->cg_exec);
    cudaGraphDestroy(g->cg);
    g->cg_exec = nullptr;
  }
  if (!g->cg_exec) {
    cudaGraph_t graph = nullptr;
    CK(cudaGraphCreate(&graph, 0));
    cudaGraphNode_t reset = nullptr, kern = nullptr;
    cudaMemsetParams mp{};
    mp.dst = g->ctl;
    mp.value = 0;
    mp.elementSize = 1;
    mp.width = sizeof(RankCtl);
    mp.height = 1;
    mp.pitch = sizeof(RankCtl);
    CK(cudaGraphAddMemsetNode(&reset, graph, nullptr, 0, &mp));
    CK(cudaGraphAddKernelNode(&kern, graph, &reset, 1, &kp));
    cudaLaunchAttributeValue coop{};
    coop.cooperative = 1;
    CK(cudaGraphKernelNodeSetAttribute(kern, cudaLaunchAttributeCooperative, &coop));
    CK(cudaGraphInstantiate(&g->cg_exec, graph, 0));
    g->cg = graph;
    g->cg_kernel = kern;
    g->cg_f32 = F32;
    g->cg_df = marking;
  } else {
    CK(cudaGraphExecKernelNodeSetParams(g->cg_exec, g->cg_kernel, &kp));
  }
  CK(cudaGraphLaunch(g->cg_exec, g->st));
  count_launch();
  return PR_OK;
}

pr_status rank_run(Graph *g, RankMode mode, pr_stats *stats) {
  pr_status rc;
  const bool marking = mode == kModeDF || mode == kModeDT || mode == kModeDFAsync;
  if (mode == kModeDFAsync && (g->teleport || g->ncomp > 1 || g->use_graph)) {
    g->err = "asynchronous Dynamic Frontier needs a single graph in self-loop mode";
    return PR_ERR_INVALID_ARG;
  }
  // Dynamic Traversal in teleport mode: a changed dead-end mass moves every rank
  const bool start_full = marking && (g->pend_all || (mode == kModeDT && g->teleport &&
                                                      (g->n_pend_src > 0 || g->n_pend_tgt > 0)));
  if (g->teleport && (rc = graph_refresh_dead(g)) != PR_OK) return rc;
  if ((rc = graph_refresh_ident(g)) != PR_OK) return rc;
  if (!g->use_graph) CK(cudaMemsetAsync(g->ctl, 0, sizeof(RankCtl), g->st));
  if (g->barrier_us > 0 && !g->use_graph) {
    // a short bounded wait for the grid barriers (tests of the time-out path)
    g->ctl_h->bar_limit_ns = 1000ull * (unsigned long long)g->barrier_us;
    CK(cudaMemcpyAsync(&g->ctl->bar_limit_ns, &g->ctl_h->bar_limit_ns, sizeof(unsigned long long),
                       cudaMemcpyHostToDevice, g->st));
  }
  if (g->ncomp > 1) {
    CK(cudaMemsetAsync(g->dRc, 0, 3ull * g->ncomp * sizeof(unsigned long long), g->st));
    CK(cudaMemsetAsync(g->comp_out, 0, 16ull * g->ncomp, g->st));
    CK(cudaMemsetAsync(g->comp_last, 0, 8ull * g->ncomp, g->st));
  }
  CK(cudaEventRecord(g->ev0, g->st));
  rc = g->f32 ? launch<true>(g, mode, start_full) : launch<false>(g, mode, start_full);
  if (rc != PR_OK) return rc;
  CK(cudaEventRecord(g->ev1, g->st));
  CK(cudaMemcpyAsync(g->ctl_h, g->ctl, offsetof(RankCtl, dR_bits), cudaMemcpyDeviceToHost, g->st));
  CK(cudaMemcpyAsync(&g->ctl_h->vproc, &g->ctl->vproc, 5 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                     g->st));
  // the per-iteration loop's state (launch count, whether it ran, its affected count)
  CK(cudaMemcpyAsync(&g->ctl_h->ticket, &g->ctl->ticket, offsetof(RankCtl, eprev) - offsetof(RankCtl, ticket),
                     cudaMemcpyDeviceToHost, g->st));
  CK(cudaStreamSynchronize(g->st));
  count_launches(g->ctl_h->launches);
  const RankCtl &h = *g->ctl_h;
  if (h.err) {
    g->err = (h.err & 1u) ? "rank kernel: a grid barrier wait timed out"
                          : "sweep kernel: a staged copy into shared memory did not complete";
    return PR_ERR_DEVICE_TIMEOUT;
  }
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
  {
    const uint32_t k = h.iterations;
    CK(cudaMemcpyAsync(g->ctl_h->t_ns, g->ctl->t_ns, sizeof(unsigned long long) * (k + 2), cudaMemcpyDeviceToHost,
                       g->st));
    CK(cudaMemcpyAsync(g->ctl_h->it_aff, g->ctl->it_aff, sizeof(uint32_t) * (k + 1), cudaMemcpyDeviceToHost, g->st));
    CK(cudaMemcpyAsync(g->ctl_h->it_kind, g->ctl->it_kind, k + 1, cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    g->trace_ms.assign(k + 1, 0.0);
    g->trace_aff.assign(k, 0);
    g->trace_kind.assign(k, 0);
    g->trace_ms[0] = (double)(h.t_ns[1] - h.t_ns[0]) * 1e-6;  // phase 0 (marking)
    for (uint32_t i = 0; i < k; i++) {
      g->trace_ms[i + 1] = (double)(h.t_ns[i + 2] - h.t_ns[i + 1]) * 1e-6;
      g->trace_aff[i] = h.it_aff[i];
      g->trace_kind[i] = h.it_kind[i];
    }
  }
  const bool full = !marking || start_full || h.full_from != 0;
  g->last_full = full;
  uint32_t fcnt[3] = {h.final_cnt[0], h.final_cnt[1], h.final_cnt[2]};
  if (h.dense_ran) {
    // the per-iteration loop's writeback listed the whole affected set in list 0
    fcnt[0] = h.aff_total;
    fcnt[1] = fcnt[2] = 0;
  }
  for (int b = 0; b < 3; b++) g->last_list_cnt[b] = marking ? fcnt[b] : 0;
  g->n_pend_src = 0;
  g->n_pend_tgt = 0;
  g->pend_all = false;
  if (g->teleport) {
    g->D_ref = h.D_final;
    g->D_ref_n = h.D_final_n;
  }
  bool all_conv = h.converged != 0;
  if (g->ncomp > 1) {
    std::vector<uint32_t> co(4ull * g->ncomp);
    std::vector<unsigned long long> cl(g->ncomp);
    CK(cudaMemcpyAsync(co.data(), g->comp_out, 16ull * g->ncomp, cudaMemcpyDeviceToHost, g->st));
    CK(cudaMemcpyAsync(cl.data(), g->comp_last, 8ull * g->ncomp, cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    all_conv = true;
    for (uint32_t c = 0; c < g->ncomp; c++) {
      pr_stats &cs = g->comp_stats[c];
      std::memset(&cs, 0, sizeof(cs));
      cs.iterations = (int32_t)co[4 * c];
      cs.converged = (int32_t)co[4 * c + 1];
      const int64_t nc = (int64_t)g->comp_first[c + 1] - g->comp_first[c];
      cs.affected_final = full ? nc : (int64_t)co[4 * c + 2];
      if (g->f32) std::memcpy(&cs.last_delta, &cl[c], 8);
      else cs.last_delta = (double)cl[c] / kOne62;
      cs.ms_rank = ms;
      all_conv = all_conv && cs.converged;
    }
  }
  if (stats) {
    const double vb = g->f32 ? 24.0 : 36.0, eb = g->f32 ? 8.0 : 12.0;
    double last = 0.0;
    if (g->f32) std::memcpy(&last, &h.last_key, 8);
    else last = (double)h.last_key / kOne62;
    stats->iterations = (int32_t)h.iterations;
    stats->converged = all_conv ? 1 : 0;
    stats->affected_final = full ? (int64_t)g->n : (int64_t)fcnt[0] + fcnt[1] + fcnt[2];
    stats->vertices_processed = (int64_t)h.vproc;
    stats->edges_processed = (int64_t)h.eproc;
    stats->bytes_algorithmic = vb * (double)h.vproc + eb * (double)h.eproc + 8.0 * (double)h.expv +
                               4.0 * (double)h.expe + 4.0 * (double)h.appended;
    stats->last_delta = last;
    stats->ms_apply = g->ms_apply;
    stats->ms_rank = ms;
  }
  g->ms_apply = 0.0;
  return PR_OK;
}

template <bool F32>
__global__ void k_set_ranks(const double *in, uint32_t n, const typename Store<F32>::A *adeg,
                            typename Store<F32>::R *R0, typename Store<F32>::R *R1, typename Store<F32>::C *C0,
                            typename Store<F32>::C *C1, const uint32_t *perm) {
  using S = Store<F32>;
  uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  typename S::R r = S::from_double(in[perm ? perm[v] : v]);  // in: the caller's numbering
  typename S::C c = S::contrib(r, adeg[v]);
  R0[v] = r;
  R1[v] = r;
  C0[v] = c;
  C1[v] = c;
}

template <bool F32>
__global__ void k_get_ranks(const typename Store<F32>::R *Rv, uint32_t n, double *out, const uint32_t *perm) {
  uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) out[perm ? perm[v] : v] = Store<F32>::to_double(Rv[v]);  // out: the caller's numbering
}

// Dead-end mass of the current ranks: exact in 64-bit mode, plain per-thread sums and an
// ordered combine in FP32 mode.  One block.
template <bool F32>
__global__ void k_dead_mass(const uint32_t *dead, uint32_t n_dead, const typename Store<F32>::R *Rv, double *out_d,
                            long long *out_n) {
  __shared__ double sd[256];
  __shared__ long long sn[256];
  double ad = 0.0;
  long long an = 0;
  for (uint32_t k = threadIdx.x; k < n_dead; k += 256) {
    if constexpr (F32) ad += (double)Rv[dead[k]];
    else an += Rv[dead[k]];
  }
  sd[threadIdx.x] = ad;
  sn[threadIdx.x] = an;
  __syncthreads();
  if (threadIdx.x == 0) {
    double td = 0.0;
    long long tn = 0;
    for (int i = 0; i < 256; i++) {
      td += sd[i];
      tn += sn[i];
    }
    *out_d = td;
    *out_n = tn;
  }
}

// Validation of ranks a caller sets: every value finite and in [0, 2], their sum at most 2.
// Ranks are a distribution (sum 1), up to the drift of methods that leave some vertices as
// they were (Dynamic Frontier); the 64-bit fixed point holds values below 2, and a mass of
// at most 2 keeps every in-edge sum (at most alpha times the mass) below that too.
// out[0] = bad values, out[1] = sum (as the bits of a double).
__global__ void k_check_ranks(const double *in, uint32_t n, unsigned long long *out) {
  __shared__ double s_sum[8];
  __shared__ uint32_t s_bad[8];
  double sum = 0.0;
  uint32_t bad = 0;
  const uint32_t nthreads = gridDim.x * blockDim.x;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += nthreads) {
    const double x = in[v];
    if (!(x >= 0.0) || !(x <= 2.0)) bad++;  // NaN, negative, or beyond the representable range
    else sum += x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s_sum[threadIdx.x >> 5] = sum;
    s_bad[threadIdx.x >> 5] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    uint32_t b = 0;
    for (int w = 0; w < 8; w++) {
      t += s_sum[w];
      b += s_bad[w];
    }
    if (b) atomicAdd(out, (unsigned long long)b);
    atomicAdd(reinterpret_cast<double *>(out + 1), t);
  }
}

pr_status rank_check(Graph *g, const double *in_d) {
  if (g->ncomp > 1) {
    // batched handle: each graph's ranks are a distribution of their own
    std::vector<double> h(g->n);
    CK(cudaMemcpyAsync(h.data(), in_d, sizeof(double) * g->n, cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    for (uint32_t c = 0; c < g->ncomp; c++) {
      double sum = 0.0;
      for (uint32_t v = g->comp_first[c]; v < g->comp_first[c + 1]; v++) {
        const double x = h[v];
        if (!(x >= 0.0) || !(x <= 2.0)) {
          g->err = "ranks must be finite and in [0, 2]";
          return PR_ERR_INVALID_ARG;
        }
        sum += x;
      }
      if (!(sum <= 2.0)) {
        g->err = "the ranks of each graph must sum to at most 2 (a distribution, up to drift)";
        return PR_ERR_INVALID_ARG;
      }
    }
    return PR_OK;
  }
  unsigned long long *dv = nullptr, hv[2] = {0, 0};
  CK(cudaMalloc((void **)&dv, sizeof(hv)));
  cudaError_t e = cudaMemsetAsync(dv, 0, sizeof(hv), g->st);
  if (e == cudaSuccess) {
    const unsigned grid = (unsigned)std::max(1, std::min((int)((g->n + 255) / 256), g->sm_count * 8));
    k_check_ranks<<<grid, 256, 0, g->st>>>(in_d, g->n, dv);
    count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(hv, dv, sizeof(hv), cudaMemcpyDeviceToHost, g->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
  cudaFree(dv);
  if (e != cudaSuccess) return cuda_fail(g, e, "check ranks");
  double sum = 0.0;
  std::memcpy(&sum, &hv[1], sizeof(double));
  if (hv[0] != 0) {
    g->err = "ranks must be finite and in [0, 2]";
    return PR_ERR_INVALID_ARG;
  }
  if (!(sum <= 2.0)) {
    g->err = "ranks must sum to at most 2 (a distribution, up to drift)";
    return PR_ERR_INVALID_ARG;
  }
  return PR_OK;
}

pr_status rank_set(Graph *g, const double *in_d) {
  unsigned grid = (g->n + 255) / 256;
  if (g->f32) {
    using S = Store<true>;
    k_set_ranks<true><<<grid, 256, 0, g->st>>>(in_d, g->n, (const S::A *)g->adeg, (S::R *)g->R[0], (S::R *)g->R[1],
                                               (S::C *)g->C[0], (S::C *)g->C[1], g->perm);
  } else {
    using S = Store<false>;
    k_set_ranks<false><<<grid, 256, 0, g->st>>>(in_d, g->n, (const S::A *)g->adeg, (S::R *)g->R[0],
                                                (S::R *)g->R[1], (S::C *)g->C[0], (S::C *)g->C[1], g->perm);
  }
  count_launch();
  CK(cudaGetLastError());
  if (g->teleport) {
    pr_status rc = graph_refresh_dead(g);
    if (rc != PR_OK) return rc;
    struct {
      double d;
      long long n;
    } *dm = nullptr, hm{};
    CK(cudaMalloc((void **)&dm, sizeof(*dm)));
    if (g->f32)
      k_dead_mass<true><<<1, 256, 0, g->st>>>(g->dead, g->n_dead, (const float *)g->R[0], &dm->d, &dm->n);
    else
      k_dead_mass<false><<<1, 256, 0, g->st>>>(g->dead, g->n_dead, (const long long *)g->R[0], &dm->d, &dm->n);
    count_launch();
    cudaError_t e = cudaMemcpyAsync(&hm, dm, sizeof(hm), cudaMemcpyDeviceToHost, g->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
    cudaFree(dm);
    if (e != cudaSuccess) return cuda_fail(g, e, "dead-end mass");
    g->D_ref = hm.d;
    g->D_ref_n = hm.n;
  }
  CK(cudaStreamSynchronize(g->st));
  return PR_OK;
}

pr_status rank_get(Graph *g, double *out_d) {
  unsigned grid = (g->n + 255) / 256;
  if (g->f32)
    k_get_ranks<true><<<grid, 256, 0, g->st>>>((const float *)g->R[0], g->n, out_d, g->perm);
  else
    k_get_ranks<false><<<grid, 256, 0, g->st>>>((const long long *)g->R[0], g->n, out_d, g->perm);
  count_launch();
  CK(cudaGetLastError());
  return PR_OK;
}

}  // namespace prdf

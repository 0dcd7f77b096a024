// sweep.cu - rank iterations as one launch each, looped on the device by a CUDA graph.
//
// Static and Naive-dynamic PageRank (Section 3.1, Section 3.3.1) and the dense iterations
// of Dynamic Frontier (Algorithm 1), its asynchronous form (Section 4.2) and Dynamic
// Traversal (Section 3.3.2) run here on single-graph handles in self-loop mode.  One
// iteration of Eq. 1 is one launch of k_sweep: no grid barrier and no loop state, so its
// register budget allows five resident blocks per SM (the persistent kernel holds four),
// and the dependent item -> column -> contribution loads of the sweep have more warps to
// overlap them.  The last block to finish an iteration reads its L-inf
// change, decides whether another iteration follows (L-inf <= tau stops, as does
// max_iter) and sets the condition of the graph's WHILE node; the host is not involved
// between iterations.
//
// The dense iterations of a Dynamic Frontier call grow the affected set in one of two
// ways, which give the same set: Algorithm 1 marks the out-neighbours of every vertex
// whose rank changed by more than tau_f, so a vertex joins iteration i + 1 exactly when
// one of its in-neighbours in G^t changed by more than tau_f in iteration i.
//   pull  every sweep item is visited; a prologue finds the vertices not yet affected
//         that have such an in-neighbour (per-vertex change flags of iteration i, kept in
//         two parities) and they join; the sweep skips vertices not affected.
//   push  the prologue scans the out-rows of the vertices whose change exceeded tau_f
//         for the first time in iteration i (as the marking launch does; later changes
//         of a vertex mark nothing new), and appends the sweep items of every newly
//         marked vertex to the compacted items, which the sweep then visits alone.
// After an iteration with many first expansions the next one pulls (its cost is about a
// full sweep, while pushing millions of out-rows costs several); otherwise it pushes (a
// few expansions without long out-rows by a plain launch, the rest by a cooperative one).
// Leaving pull for push rebuilds the compacted items, as does a set that grew by more
// than 1/16 since they were last rebuilt.  The settled compacted iterations, which need
// no prologue, run in an inner loop of the graph.  Sums are taken per vertex exactly as in the
// persistent kernel's dense sweeps, so results equal a single marking launch bit for bit.
#include <cstring>
#include <vector>

#include "rank_dev.cuh"

namespace prdf {

#ifndef PRDF_SWEEP_MIN_BLOCKS
#define PRDF_SWEEP_MIN_BLOCKS 5  // resident blocks per SM the full sweep's register budget allows
#endif
#ifndef PRDF_DF_MIN_BLOCKS
#define PRDF_DF_MIN_BLOCKS 5  // all-item Dynamic Frontier sweeps: five (some spills, measured faster than four)
#endif
constexpr int kSweepMinBlocks = PRDF_SWEEP_MIN_BLOCKS;
constexpr int kDfMinBlocks = PRDF_DF_MIN_BLOCKS;
constexpr uint32_t kPullDiv = 256;  // more than n / kPullDiv first expansions: the next iteration pulls
constexpr uint32_t kPullMin = 64;   // and at least this many
constexpr uint32_t kLightPush = 16384;  // at most this many first expansions: the light push may mark them

// Kernel parameters of k_sweep (fixed for a handle until a buffer moves; the per-call
// sizes travel in the control block).
template <bool F32>
struct SweepArgs {
  using S = Store<F32>;
  typename S::R *R0, *R1;
  typename S::C *C0, *C1;
  const typename S::A *adeg;
  const uint32_t *in_col;
  const uint2 *in_rd;
  const uint4 *items;      // all sweep items, tier order
  uint4 *items_cmp;        // the affected vertices' items (dense Dynamic Frontier); .w of a
                           // tier-0/1 item caches "out-row already marked"
  typename S::C *partials;
  uint32_t *chunk_done;
  uint16_t *stamp;
  uint32_t *bitmap;
  uint32_t *list0;
  uint32_t *xbits;
  uint32_t *xlist;
  uint8_t *emap;
  const uint2 *out_rd;     // out-row descriptors (the compacted iterations' expansion path reads lengths)
  RankCtl *ctl;
  typename S::R base;      // (1 - alpha) / n
  typename Num<F32>::B ftol;
  unsigned long long tol_key;
  uint32_t n;
  uint32_t chunk;          // edges per chunk of a tier-2 row
  int max_iter;
  cudaGraphConditionalHandle h_loop, h_pro, h_mode, h_fin;
  cudaGraphConditionalHandle h_inner;  // dense loops: the next iteration is a plain compacted one
};

// First expansions found by a dense sweep, appended to the expansion list (one atomic per
// warp round) until the iteration's entries reach cap (cap_end = the cursor where they
// would); past it a pull follows and the warp only counts them (xloc, added at the end).
__device__ __forceinline__ void note_expansion(RankCtl *ctl, uint32_t *xlist, bool push, uint32_t v, uint32_t lane,
                                               uint32_t cap_end, bool &xfull, uint32_t &xloc) {
  const uint32_t mask = __ballot_sync(kFull, push);
  if (!mask) return;
  if (xfull) {
    xloc += __popc(mask);
    return;
  }
  const uint32_t leader = __ffs(mask) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(&ctl->xcnt, (uint32_t)__popc(mask));
  base = __shfl_sync(kFull, base, leader);
  const uint32_t at = base + __popc(mask & lanemask_lt());
  if (push && at < cap_end) xlist[at] = v;
  if (base + __popc(mask) >= cap_end) xfull = true;
}

// End of an iteration, run by one thread of the last block to finish: L-inf test, the
// next iteration's way of marking (dense Dynamic Frontier), trace, loop condition.
template <bool F32, bool DF>
__device__ void sweep_decide(const SweepArgs<F32> &a, uint32_t it, bool all_items) {
  RankCtl *ctl = a.ctl;
  const unsigned long long dR = __ldcg(&ctl->dR_bits[it]);
  const uint32_t iters = it + 1;
  const bool conv = dR <= a.tol_key;
  // a prologue whose grid barrier timed out recorded an error: the loop ends
  const bool cont = !conv && (int)iters < a.max_iter && __ldcg(&ctl->err) == 0;
  ctl->iterations = iters;
  ctl->converged = conv ? 1u : 0u;
  ctl->last_key = dR;
  ctl->it_cur = iters;
  ctl->ticket = 0;
  ctl->bar = 0;  // a prologue's grid barriers count from zero
  ctl->launches += 1;
  ctl->t_ns[it + 2] = globaltimer_ns();
  if constexpr (DF) {
    uint32_t total = 0;
    for (int b = 0; b < 3; b++) {
      const uint32_t d = __ldcg(&ctl->dcnt[b]) + __ldcg(&ctl->tail[it][b]);
      ctl->dcnt[b] = d;
      ctl->final_cnt[b] = d;
      total += d;
    }
    const uint32_t jt = __ldcg(&ctl->jtotal) + __ldcg(&ctl->tail[it][3]);
    ctl->jtotal = jt;
    total += jt;
    if (!all_items) {
      // a compacted iteration swept exactly the compacted items (counted here, not by the
      // sweep: its loops keep the registers of a full sweep)
      ctl->vproc += __ldcg(&ctl->cmp_total) + __ldcg(&ctl->app_since);
      ctl->eproc += __ldcg(&ctl->cmp_edges);
    }
    ctl->eprev = __ldcg(&ctl->eproc);
    ctl->it_aff[it] = total;
    ctl->it_kind[it] = (uint8_t)__ldcg(&ctl->kind_cur);
    uint32_t pro = 0, all = 1;
    if (!cont && __ldcg(&ctl->dexpand)) {
      // the loop ends: this iteration's first expansions still mark their out-neighbours
      // (the affected set of Algorithm 1 includes the last iteration's marks), by a pull
      // over every tier when the change flags were recorded and the list may be partial,
      // by a push otherwise
      const uint32_t xend = __ldcg(&ctl->xcnt), lo = __ldcg(&ctl->xdone);
      const uint32_t x = xend - lo;
      const bool recorded = __ldcg(&ctl->erec) != 0;
      const uint32_t pull_at = max(kPullMin, a.n / kPullDiv);
      ctl->xdone = xend;
      ctl->compact_now = 0;
      ctl->push_items = 0;
      uint32_t fin = 0;
      if (x && recorded && (x > pull_at || x > __ldcg(&ctl->xcap))) {
        ctl->pull_check = 1;
        ctl->pull_all = 1;
        fin = 1;
      } else if (x) {
        ctl->push_lo = lo;
        ctl->push_n = x;
        fin = 2;
      }
      cudaGraphSetConditional(a.h_fin, fin);
    }
    if (cont) {
      const uint32_t xend = __ldcg(&ctl->xcnt), lo = __ldcg(&ctl->xdone);
      const uint32_t x = __ldcg(&ctl->dexpand) ? xend - lo : 0u;
      const bool recorded = __ldcg(&ctl->erec) != 0;
      const uint32_t pull_at = max(kPullMin, a.n / kPullDiv);
      ctl->xdone = xend;
      ctl->pull_check = 0;
      ctl->erec = 0;
      ctl->push_lo = lo;
      ctl->push_n = 0;
      ctl->compact_now = 0;
      ctl->push_items = 0;
      ctl->xcap = 0xFFFFFFFFu;
      const bool x_long = __ldcg(&ctl->x_long) != 0;
      ctl->x_long = 0;
      if (all_items && recorded && x > pull_at) {
        // many first expansions after an iteration that recorded its change flags: the next
        // iteration pulls (tiers 0 and 1 inline, tier-2 rows in a prologue); its own first
        // expansions are listed only while few enough to be pushed
        ctl->pull_check = 1;
        ctl->erec = 1;
        ctl->xcap = pull_at + 1;
        ctl->kind_cur = 7;
        pro = 1;
      } else {
        // otherwise the compacted items of the affected vertices (rebuilt when this
        // iteration swept every item: its joins are not among them), with pushed marks
        // appending their items
        ctl->push_n = x;
        ctl->compact_now = all_items ? 1u : 0u;
        ctl->push_items = all_items ? 0u : 1u;
        ctl->kind_cur = all_items ? 8u : 5u;
        pro = (x || all_items) ? 2u : 0u;
        // a few first expansions after a compacted iteration, none with a long out-row:
        // the light push (no grid barrier) marks them
        if (!all_items && x && x <= kLightPush && !x_long) pro = 3u;
        all = 0;
      }
    }
    cudaGraphSetConditional(a.h_pro, pro);
    cudaGraphSetConditional(a.h_mode, all);
    // a compacted iteration with no prologue next runs in the inner loop, whose iterations
    // have the launch cost of a full sweep's (one conditional node each)
    cudaGraphSetConditional(a.h_inner, cont && pro == 0 && all == 0 ? 1u : 0u);
  } else {
    ctl->it_aff[it] = a.n;
    ctl->it_kind[it] = 3;
    ctl->vproc += a.n;
    ctl->eproc += __ldcg(&ctl->m_cur);
  }
  if (!cont) ctl->status = kStatusDone;
  cudaGraphSetConditional(a.h_loop, cont ? 1u : 0u);
}

// Compacted iterations: v changed by more than tau_f and its cache says it may not have
// expanded yet (no bit on its tier-0/1 item, no expanded bit in the stamp of a tier-2
// row).  The stamp's expanded bit or the marking launch's bitmap decides; a first
// expansion sets the stamp bit and is appended to the expansion list (the lanes that get
// here together share one atomic; past the iteration's cap only counted), and a tier-0/1
// item gets its cache bit either way.  Out of line: after the first iteration over a
// compaction it is rare, and the sweep loops keep the registers of a full sweep.
__device__ __noinline__ void expand_cmp(RankCtl *ctl, uint16_t *stamp, const uint32_t *xbits, uint32_t *xlist,
                                        uint4 *items_cmp, const uint2 *out_rd, uint32_t v, uint32_t ci,
                                        bool has_item) {
  const uint16_t s2 = __ldcg(reinterpret_cast<const unsigned short *>(stamp + v));
  const bool was = (s2 & kStampExp) || ((__ldcg(xbits + (v >> 5)) >> (v & 31)) & 1u);
  if (!was) {
    stamp[v] = (uint16_t)(s2 | kStampExp);
    if (__ldg(&out_rd[v]).y > kInlineOut) atomicOr(&ctl->x_long, 1u);  // the next push needs the grid
  }
  if (has_item) items_cmp[ci].w = 1u;
  const uint32_t mask = __activemask();
  const uint32_t want = __ballot_sync(mask, !was);
  if (!want) return;
  const uint32_t lane = threadIdx.x & 31, leader = __ffs(want) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(&ctl->xcnt, (uint32_t)__popc(want));
  base = __shfl_sync(mask, base, leader);
  if (!was) {
    const uint32_t x0 = __ldcg(&ctl->xdone), xc = __ldcg(&ctl->xcap);
    const uint32_t cap_end = xc > 0xFFFFFFFFu - x0 ? 0xFFFFFFFFu : x0 + xc;
    const uint32_t at = base + __popc(want & lanemask_lt());
    if (at < cap_end) xlist[at] = v;
  }
}

// One iteration of Eq. 1 over sweep items.  MODE 0: every vertex (Static, Naive-dynamic).
// MODE 1: a dense Dynamic Frontier iteration over every item, vertices not affected
// skipped; when pulling, a tier-0/1 vertex not yet affected first checks its in-row
// against the previous iteration's change flags and joins if one is set (tier-2 rows were
// decided by the prologue).  MODE 2: a dense iteration over the compacted items of the
// affected vertices.  Dynamic Frontier modes record change flags when asked, and first
// expansions (changes above tau_f of vertices whose out-row was never marked from; the
// stamp's top bit then caches that it was).  Per-vertex sums are taken exactly as in the
// persistent kernel's sweeps: thread rows in runs of eight, 8-lane groups, chunk-edge
// chunks added in chunk order.
template <bool F32, int MODE>
__global__ void __launch_bounds__(kRankBlock, MODE == 1 ? kDfMinBlocks : kSweepMinBlocks) k_sweep(const SweepArgs<F32> a) {
  constexpr bool DF = MODE != 0, ALL = MODE == 1, CMP = MODE == 2;
  using S = Store<F32>;
  using R = typename S::R;
  using C = typename S::C;
  using A = typename S::A;
  using B = typename Num<F32>::B;
  __shared__ unsigned long long s_key[kWarps];
  // compacted sweeps: tier-0 tiles of the compacted affected items (32 items of a round),
  // double-buffered per warp, and their barriers
  __shared__ __align__(128) uint4 s_items[CMP ? kWarps : 1][2][32];
  __shared__ __align__(8) unsigned long long s_ibar[CMP ? kWarps : 1][2];
  RankCtl *ctl = a.ctl;
  const uint32_t tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  if (CMP && lane == 0) {
    mbar_init1(smem_addr(&s_ibar[wib][0]));
    mbar_init1(smem_addr(&s_ibar[wib][1]));
  }
  __syncwarp();
  const uint32_t nwarps = (gridDim.x * kRankBlock) >> 5, gwarp = (blockIdx.x * kRankBlock + tid) >> 5;
  const uint32_t it = __ldcg(&ctl->it_cur);
  const int par = it & 1;
  const R *Rin = par ? a.R1 : a.R0;
  const C *Cin = par ? a.C1 : a.C0;
  R *Rout = par ? a.R0 : a.R1;
  C *Cout = par ? a.C0 : a.C1;
  const uint4 *T = CMP ? a.items_cmp : a.items;
  const uint32_t *cnts = CMP ? ctl->cmp_cur : ctl->sw_all;
  const uint32_t n0 = __ldcg(cnts), n1 = __ldcg(cnts + 1), n2 = __ldcg(cnts + 2);
  const uint32_t off1 = __ldcg(&ctl->sw_off[0]), off2 = __ldcg(&ctl->sw_off[1]);
  const bool expand = DF && __ldcg(&ctl->dexpand) != 0;
  const bool pulling = ALL && __ldcg(&ctl->pull_check) != 0;
  const bool erec = ALL && __ldcg(&ctl->erec) != 0;
  uint32_t cap_end = 0;
  if (ALL) {
    const uint32_t x0 = __ldcg(&ctl->xdone), xc = __ldcg(&ctl->xcap);
    cap_end = xc > 0xFFFFFFFFu - x0 ? 0xFFFFFFFFu : x0 + xc;
  }
  bool xfull = false;
  uint32_t xloc = 0, jloc = 0;
  const uint8_t *Eprev = a.emap + (size_t)((it - 1) & 1) * a.n;  // read only when pulling (it > 0)
  uint8_t *Ecur = a.emap + (size_t)(it & 1) * a.n;
  const uint16_t itk = (uint16_t)it;
  const unsigned long long pol_cols = l2_evict_first(), pol_c = l2_evict_last();
  B my_max = 0;
  uint32_t my_v = 0, my_e = 0;

  // new rank and contribution of v; returns the change as delta bits
  auto finish = [&](uint32_t v, C sum, R rold, A ad) -> B {
    const R r = a.base + sum;
    Rout[v] = r;
    st_keep(Cout + v, S::contrib(r, ad), pol_c);
    const B dr = Num<F32>::delta(r, rold);
    my_max = dr > my_max ? dr : my_max;
    return dr;
  };
  // a vertex that joins by pull: stamp and affected bit (counted, not listed: the
  // writeback lists the affected set from the stamps)
  auto join_now = [&](uint32_t v) {
    a.stamp[v] = itk;
    atomicOr(a.bitmap + (v >> 5), 1u << (v & 31));
    jloc++;
  };
  // Dynamic Frontier bookkeeping after v's change dr: change flag (iterations that record
  // them), first-expansion test; true where v's out-row is to be marked from for the first
  // time.  st = v's stamp as read and xw its word of the bitmap of out-rows the marking
  // launch scanned (all-item iterations; a joined vertex's stamp is it and it never
  // expanded); cache = the compacted item's bit (ci = its index), the word read only where
  // no cache decides
  auto book = [&](uint32_t v, B dr, uint16_t st, bool joined, uint32_t xw, uint32_t cache, uint32_t ci) -> bool {
    if (!expand) return false;
    const bool big = dr > a.ftol;
    if (erec) Ecur[v] = big ? 1 : 0;
    if (!big) return false;
    if (ALL) {
      if (st & kStampExp) return false;
      const bool was = !joined && ((xw >> (v & 31)) & 1u);
      a.stamp[v] = (uint16_t)(st | kStampExp);
      return !was;
    }
    return false;  // compacted iterations: expand_cmp
  };

  // tier 0: one thread per vertex, 32 consecutive items per warp.  In all-item iterations
  // the stamp, the expanded word, the rank, the factor and the first eight columns are
  // loaded together (the row's loads do not wait for the stamp; a vertex not affected
  // wastes them).  These launches serve self-loop mode only, where a one-entry row is the
  // vertex's own self-loop.
  //
  // Every tier has the items of its next round on the way while it works on the current
  // one, so a round's row loads wait for no item: the next round's items are loaded into
  // registers, except in tier 0 of a compacted sweep, which stages each round's 32
  // compacted items (512 contiguous bytes) into the warp's shared-memory slot with one
  // bulk copy issued a round ahead (two slots per warp; round r uses slot r & 1 for the
  // (r >> 1)-th time, hence that phase parity).
  const uint4 zero4 = make_uint4(0, 0, 0, 0);
  const uint32_t sbar = smem_addr(&s_ibar[CMP ? wib : 0][0]), sbuf = smem_addr(&s_items[CMP ? wib : 0][0][0]);
  uint32_t rr = 0;
  auto stage = [&](uint32_t first, uint32_t cnt, uint32_t slot) {
    if (lane == 0) bulk_stage(sbuf + slot * 512u, T + first, cnt * 16u, sbar + slot * 8u);
  };
  // wait for round rr's items; on a copy that never lands, record the error, wait once
  // more (bounded) for the copies in flight and tell the tier to stop
  auto landed = [&](bool next_staged) -> bool {
    const uint32_t slot = rr & 1u;
    if (mbar_wait(sbar + slot * 8u, (rr >> 1) & 1u, kStageTimeoutNs)) return true;
    if (lane == 0) atomicOr(&ctl->err, 2u);
    mbar_wait(sbar + slot * 8u, (rr >> 1) & 1u, kStageTimeoutNs);
    if (next_staged) mbar_wait(sbar + (slot ^ 1u) * 8u, ((rr + 1) >> 1) & 1u, kStageTimeoutNs);
    return false;
  };
  auto tier0 = [&]() {
  uint4 item_nx = zero4;
  if constexpr (CMP) {
    if ((uint64_t)gwarp * 32 < n0) stage(gwarp * 32, min(32u, n0 - gwarp * 32), rr & 1u);
  } else {
    if ((uint64_t)gwarp * 32 + lane < n0) item_nx = ldcg(T + gwarp * 32 + lane);
  }
  for (uint32_t b0 = gwarp * 32; b0 < n0; b0 += nwarps * 32, rr++) {
    const uint32_t i = b0 + lane;
    bool act = false, join = false, push = false;
    uint4 item;
    if constexpr (CMP) {
      const uint32_t slot = rr & 1u;
      __syncwarp();  // the other slot was read by every lane in the previous round
      const bool nx = (uint64_t)b0 + nwarps * 32 < n0;
      if (nx) stage(b0 + nwarps * 32, min(32u, n0 - b0 - nwarps * 32), slot ^ 1u);
      if (!landed(nx)) break;
      item = i < n0 ? s_items[wib][slot][lane] : zero4;
    } else {
      item = item_nx;
      if ((uint64_t)i + nwarps * 32 < n0) item_nx = ldcg(T + i + nwarps * 32);
    }
    uint16_t st = 0;
    uint32_t xw = 0;
    R rold = (R)0;
    A ad = (A)0;
    uint4 q0 = make_uint4(0, 0, 0, 0), q1 = q0;
    if (i < n0) {
      const uint32_t v = item.x;
      if (ALL) {
        st = ldcg(a.stamp + v);
        if (expand) xw = __ldcg(a.xbits + (v >> 5));
      }
      rold = ldcg(Rin + v);
      ad = __ldg(a.adeg + v);
      if (item.z > 1 && item.z <= 8) {  // a one-entry row is v's self-loop: no column needed
        q0 = ld_cols(a.in_col + item.y, pol_cols);
        if (item.z > 4) q1 = ld_cols(a.in_col + item.y + 4, pol_cols);
      }
      act = !ALL || (st & kStampIt) <= itk;
      if (ALL && !act && pulling && item.z > 1) {
        if (item.z <= 8) {
          const uint32_t w[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
          uint32_t any = 0;  // every flag load issued at once (no chain of dependent loads)
#pragma unroll
          for (uint32_t j = 0; j < 8; j++) any |= j < item.z ? (uint32_t)__ldcg(Eprev + w[j]) : 0u;
          join = any != 0;
        } else {
          for (uint32_t j = 0; j < item.z && !join; j++) join = __ldcg(Eprev + __ldg(a.in_col + item.y + j)) != 0;
        }
        if (join) join_now(v);
      }
    }
    if (act || join) {
      const uint32_t v = item.x;
      C sum;
      if (item.z == 1) {
        // self-loop mode: the row is v's self-loop, and C[v] is contrib(R[v], A[v]) (stored
        // that way by the previous iteration), so it is recomputed from the values in hand
        sum = (C)0 + S::contrib(rold, ad);
      } else if (item.z <= 8) {  // the first round of row_sum_thread, from the columns in hand
        sum = (C)0;
        sum += gather4(Cin, q0, min(4u, item.z), pol_c);
        if (item.z > 4) sum += gather4(Cin, q1, min(4u, item.z - 4), pol_c);
      } else {
        sum = row_sum_thread(Cin, a.in_col + item.y, item.z, pol_cols, pol_c);
      }
      const B dr = finish(v, sum, rold, ad);
      if constexpr (ALL) push = book(v, dr, join ? itk : st, join, xw, item.w, i);
      if constexpr (CMP) {
        if (expand && dr > a.ftol && !item.w) expand_cmp(ctl, a.stamp, a.xbits, a.xlist, a.items_cmp, a.out_rd, v, i, true);
      }
      if constexpr (!CMP) my_v++;
      if constexpr (!CMP) my_e += item.z;
    }
    if constexpr (ALL) note_expansion(ctl, a.xlist, push, item.x, lane, cap_end, xfull, xloc);
  }
  };

  // tier 1: rows of lo < len <= group_max (<= kGroupMax) by 8-lane groups, four vertices per warp
  auto tier1 = [&]() {
      const uint32_t grp = lane >> 3, gl = lane & 7;
    uint4 item_nx = (uint64_t)gwarp * 4 + grp < n1 ? ldcg(T + off1 + gwarp * 4 + grp) : zero4;
    for (uint32_t b0 = gwarp * 4; b0 < n1; b0 += nwarps * 4) {
      const uint32_t i = b0 + grp;
      const uint4 item = item_nx;
      if ((uint64_t)i + nwarps * 4 < n1) item_nx = ldcg(T + off1 + i + nwarps * 4);
      bool act = false, join = false;
      uint16_t st = 0;
      uint32_t xw = 0;
      R rold = (R)0;
      A ad = (A)0;
      uint4 q[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
      if (i < n1) {
        if (ALL) st = ldcg(a.stamp + item.x);
        if (gl == 0) {
          rold = ldcg(Rin + item.x);
          ad = __ldg(a.adeg + item.x);
          if (ALL && expand) xw = __ldcg(a.xbits + (item.x >> 5));
        }
#pragma unroll
        for (int r = 0; r < 2; r++) {
          const uint32_t j = 4 * (gl + 8 * r);
          if (j < item.z) q[r] = ld_cols(a.in_col + item.y + j, pol_cols);
        }
        act = !ALL || (st & kStampIt) <= itk;
      }
      if (ALL && pulling) {
        bool h = false;
        if (i < n1 && !act) {
#pragma unroll
          for (int r = 0; r < 2; r++) {
            const uint32_t j = 4 * (gl + 8 * r);
            const uint32_t w[4] = {q[r].x, q[r].y, q[r].z, q[r].w};
#pragma unroll
            for (uint32_t k2 = 0; k2 < 4; k2++) h |= j + k2 < item.z && __ldcg(Eprev + w[k2]) != 0;
          }
        }
        join = ((__ballot_sync(kFull, h) >> (grp * 8)) & 0xFFu) != 0;
        if (join && gl == 0) join_now(item.x);
      }
      C sum = (C)0;
      if (act || join) {
#pragma unroll
        for (int r = 0; r < 2; r++) {
          const uint32_t j = 4 * (gl + 8 * r);
          if (j < item.z) sum += gather4(Cin, q[r], min(4u, item.z - j), pol_c);
        }
      }
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
      bool push = false;
      if ((act || join) && gl == 0) {
        const B dr = finish(item.x, sum, rold, ad);
        if constexpr (ALL) push = book(item.x, dr, join ? itk : st, join, xw, item.w, off1 + i);
        if constexpr (CMP) {
          if (expand && dr > a.ftol && !item.w)
            expand_cmp(ctl, a.stamp, a.xbits, a.xlist, a.items_cmp, a.out_rd, item.x, off1 + i, true);
        }
        if constexpr (!CMP) my_v++;
        if constexpr (!CMP) my_e += item.z;
      }
      if constexpr (ALL) note_expansion(ctl, a.xlist, push, item.x, lane, cap_end, xfull, xloc);
    }
  };

  // tier 2: chunks of at most kChunk edges dealt round-robin to warps; a row split into several chunks
  // is finished by the warp that completes its last chunk, which adds the partial sums in
  // chunk order
  C *part = a.partials;
  auto tier2 = [&]() {
  uint4 item_nx = gwarp < n2 ? ldcg(T + off2 + gwarp) : zero4;
  for (uint32_t k = gwarp; k < n2; k += nwarps) {
    const uint4 ch = item_nx;
    if ((uint64_t)k + nwarps < n2) item_nx = ldcg(T + off2 + k + nwarps);
    const uint32_t v = ch.x;
    uint16_t st = 0;
    if (ALL) st = ldcg(a.stamp + v);
    const uint32_t len = ch.z & 0x3FFu;
    const bool several = (ch.z >> 31) != 0;
    R rold = (R)0;
    A ad = (A)0;
    uint32_t deg = len, xw = 0;
    if (lane == 0) {
      rold = ldcg(Rin + v);
      ad = __ldg(a.adeg + v);
      if (several) deg = __ldg(&a.in_rd[v]).y;
      if (ALL && expand) xw = __ldcg(a.xbits + (v >> 5));
      if (CMP && expand) st = ldcg(a.stamp + v);
    }
    const uint32_t *cols = a.in_col + ch.y;
    uint4 q[4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
      const uint32_t j = 4 * (lane + 32 * r);
      if (j < len) q[r] = ld_cols(cols + j, pol_cols);
    }
    if (ALL && (st & kStampIt) > itk) continue;  // warp-uniform: not affected
    C sum = (C)0;
#pragma unroll
    for (int r = 0; r < 4; r++) {
      const uint32_t j = 4 * (lane + 32 * r);
      if (j < len) sum += gather4(Cin, q[r], min(4u, len - j), pol_c);
    }
    sum = warp_sum(sum);
    bool fin = true;
    if (several) {
      const uint32_t nch = (__shfl_sync(kFull, deg, 0) + a.chunk - 1) / a.chunk;
      uint32_t old = 0;
      if (lane == 0) {
        part[ch.w] = sum;
        __threadfence();
        old = atomicAdd(&a.chunk_done[v], 1u);
      }
      old = __shfl_sync(kFull, old, 0);
      fin = old == nch - 1;
      if (fin) {
        __threadfence();
        const uint32_t first = ch.w - ((ch.z >> 10) & 0x1FFFFFu);
        C tot = (C)0;
        for (uint32_t c = lane; c < nch; c += 32) tot += ldcg(part + first + c);
        sum = warp_sum(tot);
        if (lane == 0) a.chunk_done[v] = 0;
      }
    }
    bool push = false;
    if (fin && lane == 0) {
      const B dr = finish(v, sum, rold, ad);
      if constexpr (ALL) {
        // chunks have no cache bit: the stamp and the word read with the row decide
        if (expand) {
          const bool big = dr > a.ftol;
          if (erec) Ecur[v] = big ? 1 : 0;
          if (big && !(st & kStampExp)) {
            push = !((xw >> (v & 31)) & 1u);
            a.stamp[v] = (uint16_t)(st | kStampExp);
          }
        }
      }
      if constexpr (CMP) {
        if (expand && dr > a.ftol && !(st & kStampExp))
          expand_cmp(ctl, a.stamp, a.xbits, a.xlist, a.items_cmp, a.out_rd, v, 0, false);
      }
      if constexpr (!CMP) my_v++;
      if constexpr (!CMP) my_e += deg;
    }
    if constexpr (ALL) note_expansion(ctl, a.xlist, push, v, lane, cap_end, xfull, xloc);
  }
  };

  // Odd warps take the long rows first: their gathers, bound by the rate of random loads,
  // then overlap the latency-bound short rows of the even warps (6% less time per full
  // sweep of R-MAT scale 22 than one order for all warps)
  if (gwarp & 1) {
    tier2();
    tier0();
    tier1();
  } else {
    tier0();
    tier1();
    tier2();
  }

  // L-inf of the iteration, counters, and the last block's decision
  unsigned long long m = Num<F32>::key(my_max);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
  if (lane == 0) s_key[wib] = m;
  if constexpr (DF) {
    const unsigned long long vs = warp_sum((unsigned long long)my_v), es = warp_sum((unsigned long long)my_e);
    const uint32_t js = warp_sum(jloc);
    if (lane == 0) {
      if (vs) {
        atomicAdd(&ctl->vproc, vs);
        atomicAdd(&ctl->eproc, es);
      }
      if (xloc) atomicAdd(&ctl->xcnt, xloc);  // the same in every lane
      if (js) atomicAdd(&ctl->tail[it][3], js);
    }
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long bm = 0;
    for (int w = 0; w < kWarps; w++) bm = max(bm, s_key[w]);
    if (bm) atomicMax(&ctl->dR_bits[it], bm);
    __threadfence();
    const uint32_t t = atomicAdd(&ctl->ticket, 1u);
    if (t == gridDim.x - 1) {
      __threadfence();
      sweep_decide<F32, DF>(a, it, ALL);
    }
  }
}

// Before the first full-sweep iteration: Static starts from 1/n (both parities); the
// per-call sizes go to the control block, and the loop runs if max_iter > 0.
template <bool F32>
struct FullInit {
  using S = Store<F32>;
  typename S::R *R0, *R1;
  typename S::C *C0, *C1;
  const typename S::A *adeg;
  RankCtl *ctl;
  typename S::R init;
  uint32_t n, m, is_static;
  uint32_t sw_all[3], sw_off[2];
  int max_iter;
  cudaGraphConditionalHandle h_loop;
};

template <bool F32>
__global__ void k_full_init(const FullInit<F32> p) {
  using S = Store<F32>;
  const uint32_t nthreads = gridDim.x * blockDim.x, gtid = blockIdx.x * blockDim.x + threadIdx.x;
  if (gtid == 0 && p.ctl->t_ns[0] == 0) p.ctl->t_ns[0] = globaltimer_ns();  // unless a marking launch ran first
  if (p.is_static) {
    for (uint32_t v = gtid; v < p.n; v += nthreads) {
      const typename S::C c = S::contrib(p.init, __ldg(p.adeg + v));
      p.R0[v] = p.init;
      p.R1[v] = p.init;
      p.C0[v] = c;
      p.C1[v] = c;
    }
  }
  if (gtid == 0) {
    RankCtl *ctl = p.ctl;
    ctl->it_cur = 0;
    ctl->ticket = 0;
    for (int t = 0; t < 3; t++) ctl->sw_all[t] = p.sw_all[t];
    ctl->sw_off[0] = p.sw_off[0];
    ctl->sw_off[1] = p.sw_off[1];
    ctl->m_cur = p.m;
    ctl->status = kStatusDone;
    ctl->t_ns[1] = globaltimer_ns();
    cudaGraphSetConditional(p.h_loop, p.max_iter > 0 ? 1u : 0u);
  }
}

// After the last full-sweep iteration: both parities take the final values.
template <bool F32>
__global__ void k_full_finish(typename Store<F32>::R *R0, typename Store<F32>::R *R1, typename Store<F32>::C *C0,
                              typename Store<F32>::C *C1, uint32_t n, const RankCtl *ctl) {
  const uint32_t k = __ldcg(&ctl->iterations);
  if (k == 0) return;
  const bool fp = k & 1;
  const typename Store<F32>::R *Rf = fp ? R1 : R0;
  const typename Store<F32>::C *Cf = fp ? C1 : C0;
  typename Store<F32>::R *Ro = fp ? R0 : R1;
  typename Store<F32>::C *Co = fp ? C0 : C1;
  const uint32_t nthreads = gridDim.x * blockDim.x;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += nthreads) {
    Ro[v] = Rf[v];
    Co[v] = Cf[v];
  }
}

// Before the first dense iteration of a Dynamic Frontier (or Traversal) call: the marking
// launch left the list lengths (save_cnt, including the marks that join at next_it) and
// the iteration.  The first iteration sweeps every item with the stamp check (the marks
// for it are in place), so it needs no prologue; Dynamic Traversal records no changes and
// compacts its fixed set before the second.
struct DenseInit {
  RankCtl *ctl;
  uint32_t sw_all[3], sw_off[2];
  uint32_t n, m;
  uint32_t traversal;
  int max_iter;
  cudaGraphConditionalHandle h_loop, h_pro, h_mode, h_fin, h_inner;
};

__global__ void k_dense_init(const DenseInit p) {
  RankCtl *ctl = p.ctl;
  const uint32_t it0 = ctl->next_it;
  // per-iteration slots from it0 on start empty (a traversal's search used them for its
  // rounds; the marking launch's last marks are in save_cnt)
  for (uint32_t k = it0 + threadIdx.x; k < (uint32_t)kMaxIterLimit + 1; k += blockDim.x) {
    for (int t = 0; t < 4; t++) {
      ctl->tail[k][t] = 0;
      ctl->cmp[k][t] = 0;
    }
    ctl->hubq[k] = 0;
  }
  if (threadIdx.x == 0) {
    ctl->tail[kMaxIterLimit + 1][0] = ctl->tail[kMaxIterLimit + 1][1] = ctl->tail[kMaxIterLimit + 1][2] = 0;
    ctl->hubq[kMaxIterLimit + 1] = 0;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  ctl->it_cur = it0;
  ctl->ticket = 0;
  ctl->bar = 0;
  for (int t = 0; t < 3; t++) {
    ctl->sw_all[t] = p.sw_all[t];
    ctl->dcnt[t] = ctl->save_cnt[t];
    ctl->final_cnt[t] = ctl->save_cnt[t];
    ctl->cmp_cur[t] = 0;
  }
  ctl->sw_off[0] = p.sw_off[0];
  ctl->sw_off[1] = p.sw_off[1];
  ctl->m_cur = p.m;
  ctl->xdone = ctl->xcnt;
  ctl->xcap = max(kPullMin, p.n / kPullDiv) + 1;  // first iteration: a pull may follow
  ctl->x_long = 0;
  ctl->jtotal = 0;
  ctl->eprev = ctl->eproc;
  ctl->dense_ran = 1;
  ctl->aff_total = 0;
  ctl->cmp_total = 0;
  ctl->app_since = 0;
  ctl->push_n = 0;  // pull_check: set by a marking launch that deferred its marks to a pull
  ctl->push_items = 0;
  ctl->dmode = 1;
  ctl->compact_now = 0;
  ctl->dexpand = p.traversal ? 0u : 1u;
  ctl->erec = p.traversal ? 0u : 1u;
  ctl->kind_cur = ctl->pull_check ? 7u : 6u;
  ctl->status = kStatusDone;
  cudaGraphSetConditional(p.h_pro, 0u);
  cudaGraphSetConditional(p.h_mode, 1u);
  cudaGraphSetConditional(p.h_inner, 0u);
  if (ctl->fin_only) {
    // the marking launch ran the last iteration (recording its change flags): only its
    // marks remain, by a pull over every tier
    ctl->pull_all = 1;
    cudaGraphSetConditional(p.h_fin, 1u);
    cudaGraphSetConditional(p.h_loop, 0u);
  } else {
    ctl->iterations = it0;
    cudaGraphSetConditional(p.h_fin, 0u);
    cudaGraphSetConditional(p.h_loop, (int)it0 < p.max_iter ? 1u : 0u);
  }
}

// Prologue of a pull iteration: tier-2 rows decide their joins before the sweep.
// After the last iteration (pull_all) tier-0/1 rows pull here too, as the sweep would have.
template <bool F32>
__global__ void __launch_bounds__(kRankBlock) k_df_pull(const RankArgs<F32> a) {
  RankCtl *ctl = a.ctl;
  const uint32_t it = ldcg_u32(&ctl->it_cur);
  const uint32_t cnt0 = ldcg_u32(&ctl->dcnt[0]);
  uint32_t joined = pull_tier2(a, it, cnt0, ldcg_u32(&ctl->sw_all[2]), ldcg_u32(&ctl->sw_off[1]));
  if (ldcg_u32(&ctl->pull_all)) {
    // tier 0 and 1 rows (items before the tier-2 chunks), one thread per row
    const uint8_t *E = a.emap + (size_t)((it - 1) & 1) * a.n;
    const uint32_t n01 = ldcg_u32(&ctl->sw_off[1]), lane = threadIdx.x & 31;
    const uint32_t nthreads = gridDim.x * blockDim.x;
    for (uint32_t b0 = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; b0 < n01; b0 += nthreads) {
      const uint32_t i = b0 + lane;
      bool join = false;
      uint32_t v = 0;
      if (i < n01) {
        const uint4 item = __ldg(a.items + i);
        v = item.x;
        if (item.z > 1 && ldcg(a.stamp + v) == kNoStamp)
          for (uint32_t j = 0; j < item.z && !join; j++) join = __ldcg(E + __ldg(a.in_col + item.y + j)) != 0;
      }
      joined += pull_join(a, join, v, it, cnt0, lane);
    }
  }
  const unsigned long long s0 = warp_sum((unsigned long long)joined);
  if ((threadIdx.x & 31) == 0 && s0) atomicAdd(&ctl->appended, s0);
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&ctl->launches, 1u);
}

// Prologue of a push iteration (cooperative): the out-rows of the previous iteration's
// first expansions are marked from (the marking launch's code; long rows by the whole grid
// after a barrier), newly marked vertices appending their items to the compacted items
// when the iteration sweeps those; then, if asked or if the set grew by more than 1/16
// since, the compacted items are rebuilt from the stamps, each item's cache bit taken from
// the expanded bitmap.
template <bool F32>
__global__ void __launch_bounds__(kRankBlock, 2) k_df_push(const RankArgs<F32> a) {
  __shared__ uint32_t s_err;
  __shared__ uint32_t s_mbuf[kWarps][4 * kMarkBuf];
  RankCtl *ctl = a.ctl;
  const uint32_t tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  const uint32_t nthreads = gridDim.x * kRankBlock, gtid = blockIdx.x * kRankBlock + tid;
  const uint32_t nwarps = nthreads >> 5, gwarp = gtid >> 5;
  const uint32_t it = ldcg_u32(&ctl->it_cur);
  uint32_t epoch = 0;
  if (blockIdx.x == 0 && tid == 0) atomicAdd(&ctl->launches, 1u);
  uint32_t cnt[3];
#pragma unroll
  for (int b = 0; b < 3; b++) cnt[b] = ldcg_u32(&ctl->dcnt[b]);
  unsigned long long app = 0, xv = 0, xe = 0;
  bool compact = ldcg_u32(&ctl->compact_now) != 0;
  const bool items = ldcg_u32(&ctl->push_items) != 0;
  const uint32_t pn = ldcg_u32(&ctl->push_n);
  if (pn) {
    const uint32_t lo = ldcg_u32(&ctl->push_lo);
    WarpBuf wb{s_mbuf[wib], {0u, 0u, 0u, 0u}, false, it, items && !compact};
    for (uint32_t k0 = gwarp * 32; k0 < pn; k0 += nwarps * 32) {
      const bool p = k0 + lane < pn;
      const uint32_t x = p ? ldcg_u32(a.xlist + lo + k0 + lane) : 0u;
      const ExpandOut o = expand_lanes(a, p ? 1 : 0, x, it, cnt[0], cnt[1], cnt[2], &wb);
      app += o.app;
      xv += o.xv;
      xe += o.xe;
    }
    flush_marks(a, it, cnt, lane, wb);
    if (!grid_sync(ctl, epoch, &s_err)) return;
    if (__ldcg(&ctl->hubq[it]) != 0) {
      app += hub_pass(a, it, cnt, lane, gwarp, nwarps, wb);
      flush_marks(a, it, cnt, lane, wb);
      if (!grid_sync(ctl, epoch, &s_err)) return;
    }
    if (items && !compact && ldcg_u32(&ctl->app_since) > ldcg_u32(&ctl->cmp_total) / 16) compact = true;
  }
  if (compact) {
    // keep the items of vertices stamped <= it, one pass: a block takes rounds of 2048
    // items (eight per thread, each a coalesced warp-wide load), counts the kept ones per
    // (load, warp), reserves their places with one atomic per round and writes them in the
    // round's item order (rounds land in the order of their atomics); the stamp also sets
    // each tier-0/1 item's cache bit
    __shared__ uint32_t s_cnt[8][kWarps], s_base;
    const uint32_t seg[3][2] = {{0u, ldcg_u32(&ctl->sw_all[0])},
                                {ldcg_u32(&ctl->sw_off[0]), ldcg_u32(&ctl->sw_all[1])},
                                {ldcg_u32(&ctl->sw_off[1]), ldcg_u32(&ctl->sw_all[2])}};
    const uint32_t slot = it + 1;
    // (cmp[slot][3] sums the in-edges of the kept vertices: a chunk item's length is its
    // share of the row)
    auto kept = [&](uint32_t t, uint32_t idx, uint4 &item) -> bool {
      item = __ldg(a.items + seg[t][0] + idx);
      const uint16_t st = ldcg(a.stamp + item.x);
      const bool keep = (st & kStampIt) <= (uint16_t)it;
      if (keep && t < 2)
        item.w = ((st & kStampExp) || (__ldcg(a.xbits + (item.x >> 5)) >> (item.x & 31)) & 1u) ? 1u : 0u;
      return keep;
    };
    constexpr uint32_t kRound = 8 * kRankBlock;
    for (uint32_t t = 0; t < 3; t++) {
      const uint32_t cntt = seg[t][1];
      uint32_t e = 0;
      for (uint32_t r0 = blockIdx.x * kRound; r0 < cntt; r0 += gridDim.x * kRound) {
        uint4 item[8];
        uint32_t keepm = 0;
#pragma unroll
        for (uint32_t j = 0; j < 8; j++) {
          const uint32_t idx = r0 + j * kRankBlock + tid;
          item[j] = make_uint4(0, 0, 0, 0);
          if (idx < cntt && kept(t, idx, item[j])) {
            keepm |= 1u << j;
            e += t < 2 ? item[j].z : (item[j].z & 0x3FFu);
          }
        }
#pragma unroll
        for (uint32_t j = 0; j < 8; j++) {
          const uint32_t m = __ballot_sync(kFull, (keepm >> j) & 1u);
          if (lane == 0) s_cnt[j][wib] = __popc(m);
        }
        __syncthreads();
        if (tid == 0) {
          uint32_t tot = 0;
          for (int j = 0; j < 8; j++)
            for (int w = 0; w < kWarps; w++) {
              const uint32_t c = s_cnt[j][w];
              s_cnt[j][w] = tot;
              tot += c;
            }
          s_base = tot ? atomicAdd(&ctl->cmp[slot][t], tot) : 0u;
        }
        __syncthreads();
        const uint32_t base = s_base;
#pragma unroll
        for (uint32_t j = 0; j < 8; j++) {
          const bool k = (keepm >> j) & 1u;
          const uint32_t m = __ballot_sync(kFull, k);
          if (k) a.items_cmp[seg[t][0] + base + s_cnt[j][wib] + __popc(m & lanemask_lt())] = item[j];
        }
        __syncthreads();  // s_cnt and s_base are reused by the next round
      }
      e = warp_sum(e);
      if (lane == 0 && e) atomicAdd(&ctl->cmp[slot][3], e);
    }
    if (!grid_sync(ctl, epoch, &s_err)) return;
    if (blockIdx.x == 0 && tid == 0) {
      uint32_t total = 0;
      for (int t = 0; t < 3; t++) {
        ctl->cmp_cur[t] = __ldcg(&ctl->cmp[slot][t]);
        total += cnt[t] + __ldcg(&ctl->tail[it][t]);
      }
      ctl->cmp_total = total + __ldcg(&ctl->jtotal);
      ctl->app_since = 0;
      ctl->cmp_edges = __ldcg(&ctl->cmp[slot][3]);
      ctl->kind_cur = 8;
    }
  }
  const unsigned long long s0 = warp_sum(app), s1 = warp_sum(xv), s2 = warp_sum(xe);
  if (lane == 0) {
    if (s0) atomicAdd(&ctl->appended, s0);
    if (s1) atomicAdd(&ctl->expv, s1);
    if (s2) atomicAdd(&ctl->expe, s2);
  }
}

// Prologue of a compacted iteration after which a few vertices expanded for the first time,
// none of them with an out-row longer than kInlineOut: the warps that read them from the
// expansion list mark their out-rows and append the items of the newly marked vertices,
// with no grid barrier (the hub queue is not needed), so it costs a plain launch instead
// of a cooperative one with barriers.
template <bool F32>
__global__ void __launch_bounds__(kRankBlock, 2) k_df_push_light(const RankArgs<F32> a) {
  __shared__ uint32_t s_mbuf[kWarps][4 * kMarkBuf];
  RankCtl *ctl = a.ctl;
  const uint32_t tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  const uint32_t nwarps = (gridDim.x * kRankBlock) >> 5, gwarp = (blockIdx.x * kRankBlock + tid) >> 5;
  const uint32_t it = ldcg_u32(&ctl->it_cur);
  if (blockIdx.x == 0 && tid == 0) atomicAdd(&ctl->launches, 1u);
  uint32_t cnt[3];
#pragma unroll
  for (int b = 0; b < 3; b++) cnt[b] = ldcg_u32(&ctl->dcnt[b]);
  const uint32_t pn = ldcg_u32(&ctl->push_n), lo = ldcg_u32(&ctl->push_lo);
  WarpBuf wb{s_mbuf[wib], {0u, 0u, 0u, 0u}, false, it, true};
  unsigned long long app = 0, xv = 0, xe = 0;
  for (uint32_t k0 = gwarp * 32; k0 < pn; k0 += nwarps * 32) {
    const bool p = k0 + lane < pn;
    const uint32_t x = p ? ldcg_u32(a.xlist + lo + k0 + lane) : 0u;
    const ExpandOut o = expand_lanes(a, p ? 1 : 0, x, it, cnt[0], cnt[1], cnt[2], &wb);
    app += o.app;
    xv += o.xv;
    xe += o.xe;
  }
  flush_marks(a, it, cnt, lane, wb);
  const unsigned long long s0 = warp_sum(app), s1 = warp_sum(xv), s2 = warp_sum(xe);
  if (lane == 0) {
    if (s0) atomicAdd(&ctl->appended, s0);
    if (s1) atomicAdd(&ctl->expv, s1);
    if (s2) atomicAdd(&ctl->expe, s2);
  }
}

// Writeback of a dense Dynamic Frontier call: every affected vertex (stamp set) gets its
// final values in both parities (parity iterations & 1), its per-call marks and change
// flags are cleared, and it is listed in list 0 (each block lists its own range of
// vertices after one atomic for its offset), which is then the call's affected set.
template <bool F32>
__global__ void __launch_bounds__(256) k_df_finish(const RankArgs<F32> a) {
  using S = Store<F32>;
  using R = typename S::R;
  using C = typename S::C;
  __shared__ uint32_t s_w[8], s_base;
  RankCtl *ctl = a.ctl;
  const uint32_t tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  const bool fp = __ldcg(&ctl->iterations) & 1;
  const R *Rf = fp ? a.R1 : a.R0;
  const C *Cf = fp ? a.C1 : a.C0;
  R *Ro = fp ? a.R0 : a.R1;
  C *Co = fp ? a.C0 : a.C1;
  const uint32_t per = ((a.n + gridDim.x - 1) / gridDim.x + 255) & ~255u;
  const uint32_t lo = min(a.n, blockIdx.x * per), hi = min(a.n, lo + per);
  uint32_t c = 0;
  for (uint32_t v = lo + tid; v < hi; v += 256) c += ldcg(a.stamp + v) != kNoStamp ? 1u : 0u;
  c = warp_sum(c);
  if (lane == 0) s_w[wib] = c;
  __syncthreads();
  if (tid == 0) {
    uint32_t t = 0;
    for (int w = 0; w < 8; w++) t += s_w[w];
    s_base = t ? atomicAdd(&ctl->aff_total, t) : 0u;
  }
  __syncthreads();
  uint32_t at = s_base;
  for (uint32_t v0 = lo; v0 < hi; v0 += 256) {
    const uint32_t v = v0 + tid;
    const bool f = v < hi && ldcg(a.stamp + v) != kNoStamp;
    const uint32_t mask = __ballot_sync(kFull, f);
    __syncthreads();  // s_w free again
    if (lane == 0) s_w[wib] = __popc(mask);
    __syncthreads();
    uint32_t before = 0, all = 0;
    for (int w = 0; w < 8; w++) {
      before += w < (int)wib ? s_w[w] : 0u;
      all += s_w[w];
    }
    if (f) {
      a.list0[at + before + __popc(mask & lanemask_lt())] = v;
      Ro[v] = __ldcg(Rf + v);
      Co[v] = __ldcg(Cf + v);
      a.bitmap[v >> 5] = 0u;
      a.xbits[v >> 5] = 0u;
      a.stamp[v] = kNoStamp;
      a.emap[v] = 0;
      a.emap[a.n + v] = 0;
    }
    at += all;
  }
}

// ------------------------------------------------------------------ host side ---

namespace {

struct LoopGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t init = nullptr;
  cudaGraphConditionalHandle h_loop = 0, h_pro = 0, h_mode = 0, h_fin = 0, h_inner = 0;
  std::vector<unsigned char> key;
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    init = nullptr;
    key.clear();
  }
};

struct Loops {
  LoopGraph full;
  LoopGraph dense[2];  // synchronous, asynchronous (aliased parities)
};

template <class T>
void append_key(std::vector<unsigned char> &k, const T &x) {
  const unsigned char *p = reinterpret_cast<const unsigned char *>(&x);
  k.insert(k.end(), p, p + sizeof(T));
}

#define CKG(call)                                           \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(g, e_, #call);  \
  } while (0)

cudaError_t add_kernel(cudaGraphNode_t *node, cudaGraph_t graph, const cudaGraphNode_t *dep, size_t ndep,
                       const void *fn, dim3 grid, dim3 block, void **args, bool coop) {
  cudaKernelNodeParams kp{};
  kp.func = const_cast<void *>(fn);
  kp.gridDim = grid;
  kp.blockDim = block;
  kp.sharedMemBytes = 0;
  kp.kernelParams = args;
  cudaError_t e = cudaGraphAddKernelNode(node, graph, dep, ndep, &kp);
  if (e == cudaSuccess && coop) {
    cudaLaunchAttributeValue v{};
    v.cooperative = 1;
    e = cudaGraphKernelNodeSetAttribute(*node, cudaLaunchAttributeCooperative, &v);
  }
  return e;
}

cudaError_t add_conditional(cudaGraphNode_t *node, cudaGraph_t graph, const cudaGraphNode_t *dep, size_t ndep,
                            cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type, cudaGraph_t *body,
                            unsigned size = 1) {
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = type;
  np.conditional.size = size;
  cudaError_t e = cudaGraphAddNode(node, graph, dep, nullptr, ndep, &np);
  if (e == cudaSuccess)
    for (unsigned k = 0; k < size; k++) body[k] = np.conditional.phGraph_out[k];
  return e;
}

template <bool F32>
SweepArgs<F32> sweep_args(const Graph *g, bool async) {
  using S = Store<F32>;
  SweepArgs<F32> a{};
  a.R0 = (typename S::R *)g->R[0];
  a.R1 = (typename S::R *)(async ? g->R[0] : g->R[1]);
  a.C0 = (typename S::C *)g->C[0];
  a.C1 = (typename S::C *)(async ? g->C[0] : g->C[1]);
  a.adeg = (const typename S::A *)g->adeg;
  a.in_col = g->in.col;
  a.in_rd = g->in.rd;
  a.items = g->items;
  a.items_cmp = g->items_cmp;
  a.partials = (typename S::C *)g->partials;
  a.chunk_done = g->chunk_done;
  a.stamp = g->stamp;
  a.bitmap = g->bitmap;
  a.list0 = g->list[0];
  a.xbits = g->xbits;
  a.xlist = g->xlist;
  a.emap = g->emap;
  a.out_rd = g->out.rd;
  a.ctl = g->ctl;
  const double n = (double)g->n;
  if constexpr (F32) {
    a.base = (float)((1.0 - g->p.alpha) / n);
    float ft = (float)g->p.frontier_tol;
    std::memcpy(&a.ftol, &ft, 4);
    double tl = g->p.tol;
    std::memcpy(&a.tol_key, &tl, 8);
  } else {
    const double one = 4611686018427387904.0;  // 2^62
    a.base = std::llrint((1.0 - g->p.alpha) / n * one);
    a.ftol = (unsigned long long)std::floor(std::min(g->p.frontier_tol * one, 9.0e18));
    a.tol_key = (unsigned long long)std::floor(std::min(g->p.tol * one, 9.0e18));
  }
  a.n = g->n;
  a.chunk = g->chunk_len;
  a.max_iter = g->p.max_iter;
  return a;
}

template <bool F32>
pr_status full_impl(Graph *g, bool from_init) {
  using S = Store<F32>;
  Loops *L = (Loops *)g->loops;
  LoopGraph &lg = L->full;
  SweepArgs<F32> a = sweep_args<F32>(g, false);
  std::vector<unsigned char> key;
  append_key(key, a);
  append_key(key, g->sweep_grid);
  if (lg.exec && key != lg.key) lg.release();
  FullInit<F32> ip{};
  ip.R0 = (typename S::R *)g->R[0];
  ip.R1 = (typename S::R *)g->R[1];
  ip.C0 = (typename S::C *)g->C[0];
  ip.C1 = (typename S::C *)g->C[1];
  ip.adeg = (const typename S::A *)g->adeg;
  ip.ctl = g->ctl;
  if constexpr (F32) ip.init = (float)(1.0 / (double)g->n);
  else ip.init = std::llrint(1.0 / (double)g->n * 4611686018427387904.0);
  ip.n = g->n;
  ip.m = (uint32_t)g->m;
  ip.is_static = from_init ? 1u : 0u;
  for (int t = 0; t < 3; t++) ip.sw_all[t] = g->item_cnt[t];
  ip.sw_off[0] = g->item_cnt[0];
  ip.sw_off[1] = g->item_cnt[0] + g->item_cnt[1];
  ip.max_iter = g->p.max_iter;
  const dim3 init_grid(std::max(1, g->sm_count * 4)), init_block(256);
  if (!lg.exec) {
    CKG(cudaGraphCreate(&lg.graph, 0));
    CKG(cudaGraphConditionalHandleCreate(&lg.h_loop, lg.graph, 0, 0));
    ip.h_loop = lg.h_loop;
    a.h_loop = lg.h_loop;
    void *iargs[] = {(void *)&ip};
    CKG(add_kernel(&lg.init, lg.graph, nullptr, 0, (const void *)k_full_init<F32>, init_grid, init_block, iargs, false));
    cudaGraphNode_t wnode = nullptr, snode = nullptr, fnode = nullptr;
    cudaGraph_t body = nullptr;
    CKG(add_conditional(&wnode, lg.graph, &lg.init, 1, lg.h_loop, cudaGraphCondTypeWhile, &body));
    void *sargs[] = {(void *)&a};
    CKG(add_kernel(&snode, body, nullptr, 0, (const void *)k_sweep<F32, 0>, dim3(g->sweep_grid), dim3(kRankBlock),
                   sargs, false));
    typename S::R *R0 = ip.R0, *R1 = ip.R1;
    typename S::C *C0 = ip.C0, *C1 = ip.C1;
    uint32_t n = g->n;
    const RankCtl *ctl = g->ctl;
    void *fargs[] = {(void *)&R0, (void *)&R1, (void *)&C0, (void *)&C1, (void *)&n, (void *)&ctl};
    CKG(add_kernel(&fnode, lg.graph, &wnode, 1, (const void *)k_full_finish<F32>, init_grid, init_block, fargs,
                   false));
    CKG(cudaGraphInstantiate(&lg.exec, lg.graph, 0));
    lg.key = key;
  } else {
    ip.h_loop = lg.h_loop;
    cudaKernelNodeParams kp{};
    void *iargs[] = {(void *)&ip};
    kp.func = (void *)k_full_init<F32>;
    kp.gridDim = init_grid;
    kp.blockDim = init_block;
    kp.kernelParams = iargs;
    CKG(cudaGraphExecKernelNodeSetParams(lg.exec, lg.init, &kp));
  }
  CKG(cudaGraphLaunch(lg.exec, g->st));
  count_launches(2);  // init and writeback; the loop's launches are counted on the device
  return PR_OK;
}

template <bool F32>
pr_status dense_impl(Graph *g, RankMode mode, const RankArgs<F32> &ra_in) {
  const bool async = mode == kModeDFAsync;
  Loops *L = (Loops *)g->loops;
  LoopGraph &lg = L->dense[async ? 1 : 0];
  SweepArgs<F32> a = sweep_args<F32>(g, async);
  // the prologue's arguments without the per-call fields it does not read (copied byte for
  // byte: the cache key below compares bytes, padding included, and the caller's
  // value-initialised struct has zero padding)
  RankArgs<F32> ra;
  std::memcpy(&ra, &ra_in, sizeof ra);
  ra.it_c0 = ra.it_c1 = ra.it_c2 = 0;
  ra.n_pend_src = ra.n_pend_tgt = 0;
  ra.pend_src = ra.pend_tgt = nullptr;
  ra.n_dead = 0;
  ra.D_ref_n = 0;
  ra.D_ref_d = 0.0;
  ra.mode = 0;
  ra.start_full = 0;
  ra.split = 0;
  ra.defer_at = 0;  // depends on the edge count, which changes with every batch
  std::vector<unsigned char> key;
  append_key(key, a);
  append_key(key, ra);
  append_key(key, g->dfsweep_grid);
  append_key(key, g->cmpsweep_grid);
  append_key(key, g->pro_grid);
  if (lg.exec && key != lg.key) lg.release();
  DenseInit ip{};
  ip.ctl = g->ctl;
  for (int t = 0; t < 3; t++) ip.sw_all[t] = g->item_cnt[t];
  ip.sw_off[0] = g->item_cnt[0];
  ip.sw_off[1] = g->item_cnt[0] + g->item_cnt[1];
  ip.traversal = mode == kModeDT ? 1u : 0u;
  ip.max_iter = g->p.max_iter;
  ip.n = g->n;
  ip.m = (uint32_t)g->m;
  if (!lg.exec) {
    CKG(cudaGraphCreate(&lg.graph, 0));
    CKG(cudaGraphConditionalHandleCreate(&lg.h_loop, lg.graph, 0, 0));
    CKG(cudaGraphConditionalHandleCreate(&lg.h_fin, lg.graph, 0, 0));
    ip.h_fin = lg.h_fin;
    a.h_fin = lg.h_fin;
    cudaGraphNode_t wnode = nullptr, inode = nullptr, pnode = nullptr, fnode = nullptr;
    cudaGraph_t body = nullptr;
    ip.h_loop = lg.h_loop;
    // the WHILE node and its body first: the prologue's handle belongs to the body, and the
    // init node (added after it, then made its predecessor) sets it
    CKG(add_conditional(&wnode, lg.graph, nullptr, 0, lg.h_loop, cudaGraphCondTypeWhile, &body));
    CKG(cudaGraphConditionalHandleCreate(&lg.h_pro, body, 0, 0));
    CKG(cudaGraphConditionalHandleCreate(&lg.h_mode, body, 1, 0));
    CKG(cudaGraphConditionalHandleCreate(&lg.h_inner, body, 0, 0));
    ip.h_pro = lg.h_pro;
    ip.h_mode = lg.h_mode;
    ip.h_inner = lg.h_inner;
    a.h_loop = lg.h_loop;
    a.h_pro = lg.h_pro;
    a.h_mode = lg.h_mode;
    a.h_inner = lg.h_inner;
    // SWITCH on the prologue: 0 = none, 1 = tier-2 pull, 2 = push (and compaction), 3 = light push
    cudaGraph_t pb[4] = {nullptr, nullptr, nullptr, nullptr};
    CKG(add_conditional(&inode, body, nullptr, 0, lg.h_pro, cudaGraphCondTypeSwitch, pb, 4));
    cudaGraphNode_t enode = nullptr, pull_node = nullptr;
    CKG(cudaGraphAddEmptyNode(&enode, pb[0], nullptr, 0));
    void *pargs[] = {(void *)&ra};
    CKG(add_kernel(&pull_node, pb[1], nullptr, 0, (const void *)k_df_pull<F32>, dim3(std::max(1, g->sm_count * 8)),
                   dim3(kRankBlock), pargs, false));
    CKG(add_kernel(&pnode, pb[2], nullptr, 0, (const void *)k_df_push<F32>, dim3(g->pro_grid), dim3(kRankBlock), pargs,
                   true));
    cudaGraphNode_t lnode = nullptr;
    CKG(add_kernel(&lnode, pb[3], nullptr, 0, (const void *)k_df_push_light<F32>, dim3(std::max(1, g->sm_count)),
                   dim3(kRankBlock), pargs, false));
    // SWITCH on the iteration's mode: 0 = compacted items, 1 = every item
    cudaGraph_t sw[2] = {nullptr, nullptr};
    cudaGraphNode_t swnode = nullptr, s0 = nullptr, s1 = nullptr;
    CKG(add_conditional(&swnode, body, &inode, 1, lg.h_mode, cudaGraphCondTypeSwitch, sw, 2));
    void *sargs[] = {(void *)&a};
    CKG(add_kernel(&s0, sw[0], nullptr, 0, (const void *)k_sweep<F32, 2>, dim3(g->cmpsweep_grid), dim3(kRankBlock),
                   sargs, false));
    CKG(add_kernel(&s1, sw[1], nullptr, 0, (const void *)k_sweep<F32, 1>, dim3(g->dfsweep_grid), dim3(kRankBlock),
                   sargs, false));
    // then the run of plain compacted iterations that follows (WHILE on h_inner)
    cudaGraph_t ib = nullptr;
    cudaGraphNode_t inner = nullptr, s2 = nullptr;
    CKG(add_conditional(&inner, body, &swnode, 1, lg.h_inner, cudaGraphCondTypeWhile, &ib));
    CKG(add_kernel(&s2, ib, nullptr, 0, (const void *)k_sweep<F32, 2>, dim3(g->cmpsweep_grid), dim3(kRankBlock), sargs,
                   false));
    void *iargs[] = {(void *)&ip};
    CKG(add_kernel(&lg.init, lg.graph, nullptr, 0, (const void *)k_dense_init, dim3(1), dim3(32), iargs, false));
    cudaGraphEdgeData ed{};
    CKG(cudaGraphAddDependencies(lg.graph, &lg.init, &wnode, &ed, 1));
    // the marks of the last iteration: 0 = none, 1 = pull over every tier, 2 = push
    cudaGraph_t fb[3] = {nullptr, nullptr, nullptr};
    cudaGraphNode_t fsw = nullptr, fe = nullptr, fpull = nullptr, fpush = nullptr;
    CKG(add_conditional(&fsw, lg.graph, &wnode, 1, lg.h_fin, cudaGraphCondTypeSwitch, fb, 3));
    CKG(cudaGraphAddEmptyNode(&fe, fb[0], nullptr, 0));
    CKG(add_kernel(&fpull, fb[1], nullptr, 0, (const void *)k_df_pull<F32>, dim3(std::max(1, g->sm_count * 8)),
                   dim3(kRankBlock), pargs, false));
    CKG(add_kernel(&fpush, fb[2], nullptr, 0, (const void *)k_df_push<F32>, dim3(g->pro_grid), dim3(kRankBlock),
                   pargs, true));
    void *fargs[] = {(void *)&ra};
    CKG(add_kernel(&fnode, lg.graph, &fsw, 1, (const void *)k_df_finish<F32>, dim3(std::max(1, g->sm_count * 4)),
                   dim3(256), fargs, false));
    CKG(cudaGraphInstantiate(&lg.exec, lg.graph, 0));
    lg.key = key;
  } else {
    ip.h_loop = lg.h_loop;
    ip.h_pro = lg.h_pro;
    ip.h_mode = lg.h_mode;
    ip.h_fin = lg.h_fin;
    ip.h_inner = lg.h_inner;
    cudaKernelNodeParams kp{};
    void *iargs[] = {(void *)&ip};
    kp.func = (void *)k_dense_init;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(32);
    kp.kernelParams = iargs;
    CKG(cudaGraphExecKernelNodeSetParams(lg.exec, lg.init, &kp));
  }
  CKG(cudaGraphLaunch(lg.exec, g->st));
  count_launches(2);  // init and writeback; the loop's launches are counted on the device
  return PR_OK;
}

}  // namespace

pr_status sweep_setup(Graph *g) {
  if (!g->emap) {
    CKG(cudaMalloc((void **)&g->emap, 2ull * g->n));
    CKG(cudaMemsetAsync(g->emap, 0, 2ull * g->n, g->st));
  }
  const void *fns[2][3] = {{(const void *)k_sweep<false, 0>, (const void *)k_sweep<false, 1>, (const void *)k_sweep<false, 2>},
                           {(const void *)k_sweep<true, 0>, (const void *)k_sweep<true, 1>, (const void *)k_sweep<true, 2>}};
  int per_mode[3] = {0, 0, 0};
  for (int k = 0; k < 3; k++) {
    CKG(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_mode[k], fns[g->f32 ? 1 : 0][k], kRankBlock, 0));
    per_mode[k] = std::max(1, std::min(per_mode[k], 8));
  }
  g->sweep_grid = per_mode[0] * g->sm_count;
  g->dfsweep_grid = per_mode[1] * g->sm_count;
  g->cmpsweep_grid = per_mode[2] * g->sm_count;
  int per_sm_pro = 0;
  CKG(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm_pro, g->f32 ? (const void *)k_df_push<true> : (const void *)k_df_push<false>, kRankBlock, 0));
  g->pro_grid = std::max(1, std::min(per_sm_pro, 4)) * g->sm_count;
  if (!g->loops) g->loops = new Loops();
  return PR_OK;
}

bool sweep_eligible(const Graph *g) {
  return g->loop_sweeps && g->ncomp == 1 && !g->teleport && !g->use_graph && g->loops != nullptr;
}

pr_status sweep_full(Graph *g, bool from_init) {
  return g->f32 ? full_impl<true>(g, from_init) : full_impl<false>(g, from_init);
}

pr_status sweep_dense(Graph *g, RankMode mode, const void *rank_args) {
  return g->f32 ? dense_impl<true>(g, mode, *(const RankArgs<true> *)rank_args)
                : dense_impl<false>(g, mode, *(const RankArgs<false> *)rank_args);
}

void sweep_free(Graph *g) {
  Loops *L = (Loops *)g->loops;
  if (L) {
    L->full.release();
    L->dense[0].release();
    L->dense[1].release();
    delete L;
    g->loops = nullptr;
  }
  cudaFree(g->emap);
  g->emap = nullptr;
}

}  // namespace prdf

// rank_dev.cuh - device-side pieces shared by the rank kernels (rank.cu) and the
// per-iteration sweep kernels (sweep.cu): the rank arithmetic of each mode, the kernel
// arguments, memory-access helpers with L2 eviction policies, the bounded grid barrier,
// and the frontier marking of Algorithm 1 (push: out-rows of expanding vertices).
#pragma once

#include <cstdint>

#include "prdf_graph.cuh"

namespace prdf {


constexpr uint64_t kBarrierTimeoutNs = 4000000000ull;  // 4 s
constexpr uint64_t kStageTimeoutNs = 1000000000ull;    // 1 s: a staged copy that has not landed by then failed
constexpr int kWarps = kRankBlock / 32;
constexpr uint32_t kFull = 0xffffffffu;
constexpr uint16_t kNoStamp = 0xFFFF;
// Dense per-iteration Dynamic Frontier launches set the stamp's top bit of an affected
// vertex whose out-row has been marked from (a cache of its expanded bit: the stamp is read
// anyway); iteration numbers stay below it (max_iter <= 1000)
constexpr uint16_t kStampExp = 0x8000;
constexpr uint16_t kStampIt = 0x7FFF;
// RankCtl::status after a launch of a split call
constexpr uint32_t kStatusDone = 1;     // the call is complete (writeback done)
constexpr uint32_t kStatusDense = 2;    // the dense iterations continue in per-iteration launches from next_it
constexpr uint32_t kStatusFull = 5;     // every vertex is affected: the full-sweep iterations follow
constexpr uint32_t kInlineOut = 128;  // longer out-rows are marked by the whole grid (hub queue)
#ifndef PRDF_RANK_MIN_BLOCKS
#define PRDF_RANK_MIN_BLOCKS 4  // resident blocks per SM the register budget must allow
#endif

// Per-mode arithmetic of the kernel.  Rank changes are compared as "delta bits"
// (non-negative values that order like unsigned integers) and reduced to an L-inf key
// (uint64, same order) for the grid-wide max and the convergence test.
template <bool F32>
struct Num;

template <>
struct Num<false> {  // 64-bit fixed point, 2^-62 units
  using R = long long;
  using B = unsigned long long;
  __device__ static B delta(R r, R rold) {
    long long d = r - rold;
    return (B)(d < 0 ? -d : d);
  }
  __device__ static unsigned long long key(B d) { return d; }
};

template <>
struct Num<true> {  // float ranks; the key is the bits of the change widened to double
  using R = float;
  using B = unsigned int;
  __device__ static B delta(R r, R rold) { return __float_as_uint(fabsf(r - rold)); }
  __device__ static unsigned long long key(B d) {
    return (unsigned long long)__double_as_longlong((double)__uint_as_float(d));
  }
};

template <bool F32>
struct RankArgs {
  using S = Store<F32>;
  using R = typename S::R;
  using B = typename Num<F32>::B;
  uint32_t n;
  const uint2 *in_rd;
  const uint32_t *in_col;
  const uint2 *out_rd;
  const uint32_t *out_col;
  R *R0, *R1;
  typename S::C *C0, *C1;
  const typename S::A *adeg;
  uint32_t *bitmap;  // affected (ever marked in this call)
  uint32_t *xbits;   // out-row already scanned in this call
  uint16_t *stamp;   // iteration a vertex joins (kNoStamp = not affected)
  uint32_t *list0, *list1, *list2;
  const uint4 *items;    // sweep items in tier order (see the graph handle)
  uint4 *items_cmp;      // affected items, compacted in dense iterations
  uint32_t it_c0, it_c1, it_c2;
  typename S::C *partials;
  uint32_t *chunk_done;
  uint32_t *hub_v, *hub_base;  // hub queue of the current slot
  // batched form (ncomp > 1): component of each vertex and per-component constants
  uint32_t ncomp;
  const uint16_t *comp;
  const R *comp_base, *comp_init;
  unsigned long long *dRc;        // [3][ncomp] per-component L-inf keys, rotating by iteration
  uint32_t *comp_out;             // [ncomp][4] iterations, converged, affected
  unsigned long long *comp_last;  // [ncomp] last L-inf key
  uint32_t dense_div;
  const uint32_t *pend_src;
  uint32_t n_pend_src;
  const uint32_t *pend_tgt;
  uint32_t n_pend_tgt;
  const uint32_t *dead;
  uint32_t n_dead;
  DeadPart *dpart;        // [2][gridDim.x]
  R base;                 // (1 - alpha) / n in the rank representation
  R init;                 // 1 / n (Static start)
  B ftol;                 // tau_f as delta bits
  unsigned long long tol_key;  // tau as an L-inf key
  unsigned long long tele_frac;  // alpha / n * 2^64 (64-bit mode, teleport)
  double tele_d;          // alpha / n (FP32 mode, teleport)
  long long D_ref_n;      // dead-end mass of the previous ranks on the previous graph
  double D_ref_d;
  int max_iter;
  int mode;  // RankMode
  int teleport;
  int start_full;  // Dynamic Frontier with every vertex affected from iteration 0
  uint32_t bin_lo, bin_hi;
  uint32_t gmax, chunk;    // sweep tiers (sweep_tier) and edges per tier-2 chunk
  RankCtl *ctl;
  // split calls (single graph, self-loop mode): once the affected set is dense the marking
  // launch stops and the iterations continue in per-iteration launches (sweep.cu)
  int split;              // this call hands its dense iterations to per-iteration launches
  uint32_t defer_at;      // split calls: a sparse set larger than this defers its marks to a pull
  uint32_t *xlist;        // vertices to expand, recorded by dense sweeps (n)
  uint8_t *emap;          // [2][n] rank change above tau_f, by iteration parity (pull marking)
  const uint32_t *item_pos;  // per vertex: index of its first sweep item
};

// Neumaier's compensated summation (Neumaier 1974), for the FP32 mode's dead-end mass.
struct Neu {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double x) {
    double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x; else c += (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ void merge(double os, double oc) {
    add(os);
    c += oc;
  }
};

template <class X>
__device__ __forceinline__ X warp_sum(X x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

// ------------------------------------------------- bulk copies into shared memory ----
// A warp stages a contiguous run of sweep items (16-byte aligned, a multiple of 16 bytes)
// into its own shared-memory buffer with one cp.async.bulk issued by lane 0; completion is
// tracked by an mbarrier (arrival count 1: lane 0's arrive with the expected bytes).

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init1(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// lane 0: expect `bytes` on `bar` and copy them from global `src` to shared `dst`.  The
// buffer's previous contents were read by the warp before (a __syncwarp orders those
// reads; the proxy fence orders them before the copy's writes).
__device__ __forceinline__ void bulk_stage(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Bounded wait for the phase of `bar` with the given parity to complete; false after
// limit_ns (the caller records the error and stops using the buffer).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  uint64_t t0 = 0;
  for (uint32_t k = 0;; k++) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((k & 255) == 0) {
      const uint64_t t = globaltimer_ns();
      if (k == 0) t0 = t;
      else if (t - t0 > limit_ns) return false;
    }
  }
}

// ------------------------------------------------------------ memory access ----

__device__ __forceinline__ unsigned long long l2_evict_first() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ unsigned long long l2_evict_last() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// Four column ids of a 16-byte aligned run (read-only during the kernel).
__device__ __forceinline__ uint4 ld_cols(const uint32_t *p, unsigned long long pol) {
  uint4 r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p), "l"(pol));
  return r;
}
// Contribution gathers.  C of the iteration's input parity is not written during the
// iteration, and a kernel boundary or the grid barrier's acquire orders every block after
// all writes of the previous iteration, so the gathers may be served by L1 (the default).
// Under the internal breadth-first numbering the short rows that one warp sweeps gather
// from nearby contributions, and L1-allocating gathers make a scale-22 R-MAT full sweep 2%
// faster in 64-bit mode and 5% in FP32 than L2-only ones (PRDF_GATHER_L2_ONLY=1), which
// were ahead under a random numbering.  (The asynchronous form reads C while it is
// written; a line that L1 still holds gives an older value, which that form allows.)
#ifndef PRDF_GATHER_L2_ONLY
#define PRDF_GATHER_L2_ONLY 0
#endif
#if PRDF_GATHER_L2_ONLY
#define PRDF_GATHER_COP "cg"
#else
#define PRDF_GATHER_COP "ca"
#endif
__device__ __forceinline__ long long ld_keep(const long long *p, unsigned long long pol) {
  long long r;
  asm("ld.global." PRDF_GATHER_COP ".L2::cache_hint.b64 %0, [%1], %2;" : "=l"(r) : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ float ld_keep(const float *p, unsigned long long pol) {
  float r;
  asm("ld.global." PRDF_GATHER_COP ".L2::cache_hint.f32 %0, [%1], %2;" : "=f"(r) : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ void st_keep(long long *p, long long v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.b64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_keep(float *p, float v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
}

__device__ __forceinline__ long long ldcg(const long long *p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg(const float *p) { return __ldcg(p); }
__device__ __forceinline__ uint32_t ldcg(const uint32_t *p) { return __ldcg(p); }
__device__ __forceinline__ uint32_t ldcg_u32(const uint32_t *p) { return __ldcg(p); }
__device__ __forceinline__ uint16_t ldcg(const uint16_t *p) {
  return __ldcg(reinterpret_cast<const unsigned short *>(p));
}

// Grid-wide barrier with a bounded wait.  Returns false (in every thread of the block)
// if the device control block holds an error.
__device__ __forceinline__ bool grid_sync(RankCtl *ctl, uint32_t &epoch, uint32_t *s_err) {
  __syncthreads();
  epoch++;
  if (threadIdx.x == 0) {
    __threadfence();
    red_release_add_u32(&ctl->bar, 1u);
    const uint32_t target = epoch * gridDim.x;
    uint64_t t0 = 0;
    uint32_t spins = 0;
    // the default limit is checked every 128 spins; a short limit set for tests, every spin
    const unsigned long long lim = *(volatile unsigned long long *)&ctl->bar_limit_ns;
    const uint32_t every = lim ? 0u : 127u;
    while (ld_acquire_u32(&ctl->bar) < target) {
      if (*(volatile uint32_t *)&ctl->err) break;
      __nanosleep(32);
      if ((++spins & every) == 0) {
        uint64_t t = globaltimer_ns();
        if (t0 == 0) {
          t0 = t;
        } else if (t - t0 > (lim ? lim : kBarrierTimeoutNs)) {
          atomicExch(&ctl->err_where, epoch);
          atomicOr(&ctl->err, 1u);
          break;
        }
      }
    }
    __threadfence();
    *s_err = *(volatile uint32_t *)&ctl->err;
  }
  __syncthreads();
  return *s_err == 0;
}

__device__ __forceinline__ int bin_of(uint32_t deg, uint32_t lo, uint32_t hi) {
  return deg <= lo ? 0 : (deg <= hi ? 1 : 2);
}

// Newly marked vertices are buffered per warp in shared memory, one run per bin, and
// appended to the bin's list with one global atomic per run rather than one per marking
// round (the list tails are contended by every warp of the grid).  Every buffer is flushed
// before the grid barrier after which the tails are read.  In dense iterations all marks
// go to list 0 and the in-degree lookup for the bin is skipped: later iterations are dense
// too (the affected set only grows) and sweep the sweep items, and the writeback only
// needs every affected vertex in some list.
constexpr uint32_t kMarkBuf = 64;
struct WarpBuf {
  uint32_t *buf;   // [4][kMarkBuf] entries of this warp's shared memory: bins 0-2, expansions
  uint32_t n[4];   // entries held per run (the same in every lane)
  bool dense;
  uint32_t slot;   // iteration the queued expansions' marks join (their count per slot)
  bool items;      // also append the marked vertices' sweep items to the compacted items
};

// Dense Dynamic Frontier iterations over compacted items: the sweep items of vertices
// marked since the items were compacted are appended to the compacted tier segments (one
// item per vertex in tiers 0 and 1, all chunks of a tier-2 row), so those iterations sweep
// exactly the affected vertices without compacting again.  Called by a whole warp with a
// run of k marked vertices.
template <bool F32>
__device__ __noinline__ void append_items(const RankArgs<F32> &a, const uint32_t *run, uint32_t k, uint32_t lane) {
  const uint32_t seg[3] = {0u, ldcg_u32(&a.ctl->sw_off[0]), ldcg_u32(&a.ctl->sw_off[1])};
  for (uint32_t i0 = 0; i0 < k; i0 += 32) {
    const uint32_t i = i0 + lane;
    uint32_t t = 3, cw = 0, pos = 0, d = 0;
    if (i < k) {
      const uint32_t w = run[i];
      d = __ldg(&a.in_rd[w]).y;
      t = (uint32_t)sweep_tier(d, a.bin_lo, a.gmax);
      cw = t == 2 ? (d + a.chunk - 1) / a.chunk : 1u;
      pos = __ldg(&a.item_pos[w]);
    }
#pragma unroll
    for (uint32_t tt = 0; tt < 3; tt++) {
      const uint32_t c = t == tt ? cw : 0u;
      uint32_t incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= (uint32_t)o) incl += y;
      }
      const uint32_t tot = __shfl_sync(kFull, incl, 31);
      if (tot == 0) continue;
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(&a.ctl->cmp_cur[tt], tot);
      base = __shfl_sync(kFull, base, 0);
      for (uint32_t c2 = 0; c2 < c; c2++) a.items_cmp[seg[tt] + base + incl - c + c2] = __ldg(a.items + pos + c2);
    }
    const uint32_t m = __ballot_sync(kFull, i < k);
    const unsigned long long de = warp_sum((unsigned long long)d);
    if (lane == 0) {
      atomicAdd(&a.ctl->app_since, (uint32_t)__popc(m));
      atomicAdd(&a.ctl->cmp_edges, de);
    }
  }
}

template <bool F32>
__device__ __forceinline__ void flush_bin(const RankArgs<F32> &a, int bb, uint32_t slot, const uint32_t cnt[3],
                                          uint32_t lane, WarpBuf &wb) {
  __syncwarp();
  const uint32_t k = wb.n[bb];
  if (k) {
    uint32_t *lists[3] = {a.list0, a.list1, a.list2};
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&a.ctl->tail[slot][bb], k);
    base = __shfl_sync(kFull, base, 0);
    for (uint32_t i = lane; i < k; i += 32) lists[bb][cnt[bb] + base + i] = wb.buf[bb * kMarkBuf + i];
    if (wb.items) append_items(a, wb.buf + bb * kMarkBuf, k, lane);
  }
  __syncwarp();
  wb.n[bb] = 0;
}

// Vertices a dense or full sweep found to expand, appended to the call's expansion list
// (each vertex at most once per call: first_expansion) in runs; the grid scans their
// out-rows after the iteration's barrier, so the sweep loops carry no marking code.
template <bool F32>
__device__ __forceinline__ void flush_expansions(const RankArgs<F32> &a, uint32_t lane, WarpBuf &wb) {
  __syncwarp();
  const uint32_t k = wb.n[3];
  if (k) {
    uint32_t base = 0;
    if (lane == 0) {
      base = atomicAdd(&a.ctl->xcnt, k);
      atomicAdd(&a.ctl->xit[wb.slot], k);
    }
    base = __shfl_sync(kFull, base, 0);
    for (uint32_t i = lane; i < k; i += 32) a.xlist[base + i] = wb.buf[3 * kMarkBuf + i];
  }
  __syncwarp();
  wb.n[3] = 0;
}

template <bool F32>
__device__ __forceinline__ void queue_expansion(const RankArgs<F32> &a, bool push, uint32_t v, uint32_t lane,
                                                WarpBuf &wb) {
  const uint32_t mask = __ballot_sync(kFull, push);
  if (mask) {
    if (wb.n[3] + __popc(mask) > kMarkBuf) flush_expansions(a, lane, wb);
    if (push) wb.buf[3 * kMarkBuf + wb.n[3] + __popc(mask & lanemask_lt())] = v;
    wb.n[3] += __popc(mask);
  }
}

template <bool F32>
__device__ __forceinline__ void flush_marks(const RankArgs<F32> &a, uint32_t slot, const uint32_t cnt[3],
                                            uint32_t lane, WarpBuf &wb) {
#pragma unroll
  for (int bb = 0; bb < 3; bb++) flush_bin(a, bb, slot, cnt, lane, wb);
  flush_expansions(a, lane, wb);
}

// Appends w where fresh to its bin's run in the warp's buffer.  Called by a whole warp.
template <bool F32>
__device__ __forceinline__ void append_mark(const RankArgs<F32> &a, bool fresh, uint32_t w, uint32_t slot,
                                            const uint32_t cnt[3], uint32_t lane, WarpBuf &wb) {
  int bin = -1;
  if (fresh) bin = wb.dense ? 0 : bin_of(__ldg(&a.in_rd[w]).y, a.bin_lo, a.bin_hi);
  const int nb = wb.dense ? 1 : 3;
  for (int bb = 0; bb < nb; bb++) {
    const uint32_t mask = __ballot_sync(kFull, bin == bb);
    if (mask) {
      if (wb.n[bb] + __popc(mask) > kMarkBuf) flush_bin(a, bb, slot, cnt, lane, wb);
      if (bin == bb) wb.buf[bb * kMarkBuf + wb.n[bb] + __popc(mask & lanemask_lt())] = w;
      wb.n[bb] += __popc(mask);
    }
  }
}

// Marks w (where valid) for iteration `slot`: a plain read of the bitmap first, then the
// atomic; a newly marked vertex is stamped and appended through the warp's buffer.  Called
// by a whole warp; returns 1 where this lane marked a new vertex.
template <bool F32>
__device__ __forceinline__ uint32_t mark_one(const RankArgs<F32> &a, bool valid, uint32_t w, uint32_t slot,
                                             const uint32_t cnt[3], uint32_t lane, WarpBuf &wb) {
  bool fresh = false;
  if (valid) {
    uint32_t bit = 1u << (w & 31);
    uint32_t *word = a.bitmap + (w >> 5);
    if (!(ldcg(word) & bit)) {
      uint32_t old = atomicOr(word, bit);
      if (!(old & bit)) {
        fresh = true;
        a.stamp[w] = (uint16_t)slot;
      }
    }
  }
  append_mark(a, fresh, w, slot, cnt, lane, wb);
  return fresh ? 1u : 0u;
}

// Marks cols[first + 32 k + lane] (k = 0, 1, ...; stride `stride`), stamping newly marked
// vertices with `slot` (the iteration they join).  Called by a whole warp.
template <bool F32>
__device__ __forceinline__ uint32_t warp_mark_range(const RankArgs<F32> &a, const uint32_t *cols, uint32_t len,
                                                    uint32_t first, uint32_t stride, uint32_t slot,
                                                    const uint32_t cnt[3], uint32_t lane, WarpBuf &wb) {
  uint32_t newly_total = 0;
  for (uint32_t j0 = first; j0 < len; j0 += stride) {
    const uint32_t j = j0 + lane;
    const bool valid = j < len;
    newly_total += mark_one(a, valid, valid ? __ldg(cols + j) : 0u, slot, cnt, lane, wb);
  }
  return newly_total;
}

// Short out-rows (at most kThreadOut entries; a row starts 16-byte aligned and its slots
// come in whole groups of four): every lane in `mine` marks its own row.  The bitmap words
// of all its entries are read together and the atomics for the clear bits are issued
// together, so a row costs two dependent round trips rather than a pair per entry; the
// stamps and warp-aggregated appends follow entry by entry.  Called by a whole warp.
constexpr uint32_t kThreadOut = 8;
template <bool F32>
__device__ __forceinline__ uint32_t lane_mark_rows(const RankArgs<F32> &a, bool mine, uint2 od, uint32_t slot,
                                                   const uint32_t cnt[3], uint32_t lane, WarpBuf &wb) {
  const uint32_t len = mine ? od.y : 0u;
  const uint32_t rounds = __reduce_max_sync(kFull, len);
  uint4 q0 = make_uint4(0, 0, 0, 0), q1 = q0;
  if (len > 0) q0 = __ldg(reinterpret_cast<const uint4 *>(a.out_col + od.x));
  if (len > 4) q1 = __ldg(reinterpret_cast<const uint4 *>(a.out_col + od.x + 4));
  const uint32_t w[kThreadOut] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
  uint32_t word[kThreadOut];
#pragma unroll
  for (uint32_t k = 0; k < kThreadOut; k++) word[k] = k < len ? ldcg(a.bitmap + (w[k] >> 5)) : ~0u;
  uint32_t fresh = 0;  // bit k: entry k newly marked by this lane
#pragma unroll
  for (uint32_t k = 0; k < kThreadOut; k++) {
    const uint32_t bit = 1u << (w[k] & 31);
    if (!(word[k] & bit) && !(atomicOr(a.bitmap + (w[k] >> 5), bit) & bit)) fresh |= 1u << k;
  }
  uint32_t newly = 0;
#pragma unroll
  for (uint32_t k = 0; k < kThreadOut; k++) {
    if (k < rounds) {
      const bool f = (fresh >> k) & 1u;
      if (f) a.stamp[w[k]] = (uint16_t)slot;
      append_mark(a, f, w[k], slot, cnt, lane, wb);
      newly += f ? 1u : 0u;
    }
  }
  return newly;
}

// True the first time v asks (per call): its out-row is then scanned by the caller.  A
// plain read first, so a vertex that keeps changing costs one load per iteration, not an
// atomic.
__device__ __forceinline__ bool first_expansion(uint32_t *xbits, uint32_t v) {
  uint32_t bit = 1u << (v & 31);
  if (__ldcg(xbits + (v >> 5)) & bit) return false;
  return !(atomicOr(xbits + (v >> 5), bit) & bit);
}
// The same with the word read beforehand (issued with the row's loads, so the test adds no
// round trip); the atomic still decides, so a stale word only costs an atomic.
__device__ __forceinline__ bool first_expansion_pre(uint32_t *xbits, uint32_t v, uint32_t word) {
  uint32_t bit = 1u << (v & 31);
  if (word & bit) return false;
  return !(atomicOr(xbits + (v >> 5), bit) & bit);
}

// Marks the out-neighbours of v for iteration `slot`: short out-rows by the calling warp,
// long ones queued for the cooperative pass that follows the iteration's barrier (entry
// index and chunk base are reserved by one 64-bit atomic, so bases ascend with the index).
// Called by a whole warp; returns the vertices this warp newly marked.
template <bool F32>
__device__ __forceinline__ uint32_t expand_vertex(const RankArgs<F32> &a, uint32_t v, uint2 od, uint32_t slot,
                                                  const uint32_t cnt[3], uint32_t lane, WarpBuf &wb) {
  if (od.y <= kInlineOut) return warp_mark_range(a, a.out_col + od.x, od.y, 0, 32, slot, cnt, lane, wb);
  if (lane == 0) {
    const uint32_t nch = (od.y + kChunk - 1) / kChunk;
    const unsigned long long old = atomicAdd(&a.ctl->hubq[slot], (1ull << 32) | nch);
    const uint32_t e = (uint32_t)(old >> 32);
    a.hub_v[e] = v;
    a.hub_base[e] = (uint32_t)old;
  }
  return 0;
}

// The cooperative pass over the queued long out-rows of `slot`: kChunk-entry chunks
// dealt round-robin to all warps of the grid.
template <bool F32>
__device__ uint32_t hub_pass(const RankArgs<F32> &a, uint32_t slot, const uint32_t cnt[3], uint32_t lane,
                             uint32_t gwarp, uint32_t nwarps, WarpBuf &wb) {
  const unsigned long long hq = __ldcg(&a.ctl->hubq[slot]);
  const uint32_t ne = (uint32_t)(hq >> 32), K = (uint32_t)hq;
  uint32_t newly = 0;
  for (uint32_t k = gwarp; k < K; k += nwarps) {
    uint32_t lo = 0, hi = ne;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (__ldcg(a.hub_base + mid) <= k) lo = mid; else hi = mid;
    }
    const uint32_t v = __ldcg(a.hub_v + lo), c = k - __ldcg(a.hub_base + lo);
    const uint2 od = __ldg(&a.out_rd[v]);
    const uint32_t start = c * kChunk;
    newly += warp_mark_range(a, a.out_col + od.x + start, min(kChunk, od.y - start), 0, 32, slot, cnt, lane, wb);
  }
  return newly;
}

template <class C>
__device__ __forceinline__ C gather4(const C *Cv, uint4 q, uint32_t valid, unsigned long long pol) {
  C s = (C)0;
  if (valid > 0) s += ld_keep(Cv + q.x, pol);
  if (valid > 1) s += ld_keep(Cv + q.y, pol);
  if (valid > 2) s += ld_keep(Cv + q.z, pol);
  if (valid > 3) s += ld_keep(Cv + q.w, pol);
  return s;
}

// Sum of C over one whole row by one thread: runs of 8 columns, all loads of a run in
// flight together.
template <class C>
__device__ __forceinline__ C row_sum_thread(const C *Cv, const uint32_t *cols, uint32_t len,
                                            unsigned long long pol_cols, unsigned long long pol_c) {
  C sum = (C)0;
  for (uint32_t j0 = 0; j0 < len; j0 += 8) {
    uint4 q[2];
#pragma unroll
    for (int k = 0; k < 2; k++)
      if (j0 + 4 * k < len) q[k] = ld_cols(cols + j0 + 4 * k, pol_cols);
#pragma unroll
    for (int k = 0; k < 2; k++)
      if (j0 + 4 * k < len) sum += gather4(Cv, q[k], min(4u, len - j0 - 4 * k), pol_c);
  }
  return sum;
}


// Dead-end mass accumulator: exact integer in 64-bit mode, Neumaier pair in FP32 mode.
template <bool F32>
struct Mass;
template <>
struct Mass<false> {
  long long s = 0;
  __device__ void add(long long x) { s += x; }
};
template <>
struct Mass<true> {
  Neu n;
  __device__ void add(double x) { n.add(x); }
};

template <bool F32>
struct Iter {
  bool full;
  typename Store<F32>::R tele;  // alpha D / n in the rank representation
};

// Rank of v from its in-edge sum, given R[v] and A[v] loaded beforehand; writes the new
// rank and contribution; returns the delta bits of |r - R[v]|.
template <bool F32>
__device__ __forceinline__ typename Num<F32>::B finish_vertex(const RankArgs<F32> &a, typename Store<F32>::R *Rout,
                                                              typename Store<F32>::C *Cout, uint32_t v,
                                                              typename Store<F32>::C sum, typename Store<F32>::R rold,
                                                              typename Store<F32>::A ad, const Iter<F32> &I,
                                                              Mass<F32> &dacc, unsigned long long pol_c,
                                                              typename Store<F32>::R base) {
  using S = Store<F32>;
  using R = typename S::R;
  R r = base + sum;
  if (a.teleport) r += I.tele;
  Rout[v] = r;
  st_keep(Cout + v, S::contrib(r, ad), pol_c);
  if (a.teleport && ad == (typename S::A)0) {
    if constexpr (F32) dacc.add(I.full ? (double)r : (double)r - (double)rold);
    else dacc.add(I.full ? r : r - rold);
  }
  return Num<F32>::delta(r, rold);
}

__device__ __forceinline__ uint4 ldcg(const uint4 *p) { return __ldcg(p); }

// Frontier expansion of the lanes' vertices that changed by more than tau_f (push):
// short out-rows by their own lanes, medium ones flattened across the warp, hub rows
// queued for the grid.  Out of line: it runs only when some lane of the warp expands, and
// keeping its registers out of the sweep loops keeps those loops free of spills.  Called
// by a whole warp.
struct ExpandOut {
  uint32_t app, xv, xe;  // vertices appended; vertices and out-edges expanded (this lane)
};
template <bool F32>
__device__ __noinline__ ExpandOut expand_lanes(const RankArgs<F32> &a, int push, uint32_t v, uint32_t slot,
                                               uint32_t c0, uint32_t c1, uint32_t c2, WarpBuf *wbp) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t cnt[3] = {c0, c1, c2};
  WarpBuf wb = *wbp;
  ExpandOut o{0u, 0u, 0u};
  uint2 od = make_uint2(0, 0);
  if (push) od = __ldg(&a.out_rd[v]);
  // short rows: each lane its own
  const bool mine = push && od.y <= kThreadOut;
  if (__any_sync(kFull, mine)) o.app += lane_mark_rows(a, mine, od, slot, cnt, lane, wb);
  // medium rows: the rows of all such lanes flattened into one run of entries, marked 128
  // at a time (four per lane; the column loads, bitmap reads and atomics of a round are in
  // flight together), so the warp spends ceil(total / 128) rounds instead of one round per
  // 32 entries of every row in turn
  const bool med = push && od.y > kThreadOut && od.y <= kInlineOut;
  const uint32_t mlen = med ? od.y : 0u;
  uint32_t incl = mlen;
#pragma unroll
  for (int k = 1; k < 32; k <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, incl, k);
    if (lane >= (uint32_t)k) incl += y;
  }
  const uint32_t total = __shfl_sync(kFull, incl, 31);
  const uint32_t excl = incl - mlen;
  for (uint32_t e0 = 0; e0 < total; e0 += 128) {
    uint32_t w[4], word[4];
    bool valid[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint32_t e = e0 + 32u * k + lane;
      // the lane whose run [excl, incl) holds entry e
      uint32_t owner = 0;
#pragma unroll
      for (uint32_t step = 16; step > 0; step >>= 1) {
        const uint32_t probe = __shfl_sync(kFull, incl, owner + step - 1);
        if (probe <= e) owner += step;
      }
      const uint32_t base = __shfl_sync(kFull, od.x, owner & 31u);
      const uint32_t first = __shfl_sync(kFull, excl, owner & 31u);
      valid[k] = e < total;
      w[k] = valid[k] ? __ldg(a.out_col + base + (e - first)) : 0u;
    }
#pragma unroll
    for (int k = 0; k < 4; k++) word[k] = valid[k] ? ldcg(a.bitmap + (w[k] >> 5)) : ~0u;
    uint32_t fresh = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint32_t bit = 1u << (w[k] & 31);
      if (!(word[k] & bit) && !(atomicOr(a.bitmap + (w[k] >> 5), bit) & bit)) fresh |= 1u << k;
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const bool f = (fresh >> k) & 1u;
      if (f) a.stamp[w[k]] = (uint16_t)slot;
      append_mark(a, f, w[k], slot, cnt, lane, wb);
      o.app += f ? 1u : 0u;
    }
  }
  if (mine || med) {
    o.xv++;
    o.xe += od.y;
  }
  // hub rows: queued for the grid
  uint32_t mask = __ballot_sync(kFull, push && od.y > kInlineOut);
  while (mask) {
    const uint32_t src = __ffs(mask) - 1;
    mask &= mask - 1;
    const uint32_t x = __shfl_sync(kFull, v, src);
    const uint2 ox = make_uint2(__shfl_sync(kFull, od.x, src), __shfl_sync(kFull, od.y, src));
    o.app += expand_vertex(a, x, ox, slot, cnt, lane, wb);
    if (lane == 0) {
      o.xv++;
      o.xe += ox.y;
    }
  }
  *wbp = wb;
  return o;
}

// One vertex's out-row (hub rows queued), by the whole warp; out of line like expand_lanes.
template <bool F32>
__device__ __noinline__ ExpandOut expand_one(const RankArgs<F32> &a, uint32_t v, uint32_t slot, uint32_t c0,
                                             uint32_t c1, uint32_t c2, WarpBuf *wbp) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t cnt[3] = {c0, c1, c2};
  WarpBuf wb = *wbp;
  const uint2 od = __ldg(&a.out_rd[v]);
  ExpandOut o{expand_vertex(a, v, od, slot, cnt, lane, wb), 0u, 0u};
  if (lane == 0) {
    o.xv = 1;
    o.xe = od.y;
  }
  *wbp = wb;
  return o;
}

// Marks for a pull iteration (called by a whole warp): stamps, affected bit, list 0.
template <bool F32>
__device__ __forceinline__ uint32_t pull_join(const RankArgs<F32> &a, bool join, uint32_t v, uint32_t it,
                                              uint32_t cnt0, uint32_t lane) {
  if (join) {
    a.stamp[v] = (uint16_t)it;
    atomicOr(a.bitmap + (v >> 5), 1u << (v & 31));
  }
  const uint32_t mask = __ballot_sync(kFull, join);
  if (mask) {
    const uint32_t leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&a.ctl->tail[it][0], (uint32_t)__popc(mask));
    base = __shfl_sync(kFull, base, leader);
    if (join) a.list0[cnt0 + base + __popc(mask & lanemask_lt())] = v;
  }
  return (uint32_t)__popc(mask);
}

// The pull of iteration it for tier-2 rows (longer than the group limit; all2 chunk items from
// items[off2]): a row not yet affected joins if an in-neighbour's change exceeded tau_f in
// iteration it - 1.  Its chunks go to several warps, so the warp of the first chunk
// decides for the row before the sweep.  Tier-0/1 rows are pulled inline by the sweep.
// Out of line: once per pull iteration.
template <bool F32>
__device__ __noinline__ uint32_t pull_tier2(const RankArgs<F32> &a, uint32_t it, uint32_t cnt0, uint32_t all2,
                                           uint32_t off2) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5, gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint8_t *E = a.emap + (size_t)((it - 1) & 1) * a.n;
  uint32_t joined = 0;
  for (uint32_t k = gwarp; k < all2; k += nwarps) {
    const uint4 ch = __ldg(a.items + off2 + k);
    const uint32_t v = ch.x;
    if (((ch.z >> 10) & 0x1FFFFFu) != 0 || ldcg(a.stamp + v) != kNoStamp) continue;  // warp-uniform
    const uint2 d = __ldg(&a.in_rd[v]);
    bool any = false;
    for (uint32_t j0 = 0; j0 < d.y && !any; j0 += 32) {
      const uint32_t j = j0 + lane;
      const bool h = j < d.y && __ldcg(E + __ldg(a.in_col + d.x + j)) != 0;
      any = __any_sync(kFull, h);
    }
    joined += pull_join(a, lane == 0 && any, v, it, cnt0, lane);
  }
  return joined;
}

}  // namespace prdf

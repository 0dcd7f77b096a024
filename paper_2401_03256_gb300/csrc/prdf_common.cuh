// prdf_common.cuh - internal declarations of the GB300 Dynamic Frontier PageRank library.
//
// Graph storage is a "slack-row" paired CSR: for each adjacency (in-edges, out-edges)
// row v is described by rd[v] = {start, len} into one column array, rows are kept
// sorted, every row starts on a 16-byte boundary (start % 4 == 0) and owns cap[v] >= len
// slots, so a batch update rewrites only the rows it touches (in place while they fit,
// otherwise the row moves to the free tail of the column array).  The packed canonical
// CSR is produced on demand by pr_get_csr.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace prdf {

constexpr int kMaxIterLimit = 1000;       // hard cap on max_iter (control arrays are sized by it)
constexpr uint64_t kSentinel = ~0ull;     // key of a dropped pair
constexpr int kRankBlock = 256;           // threads per block of the rank kernel
constexpr uint32_t kSmallSort = 4096;     // largest key count sorted by one block
constexpr uint32_t kChunk = 512;          // entries per chunk of a long row (hub out-rows; the most a sweep chunk holds)
constexpr uint32_t kGroupMax = 64;        // the longest row an 8-lane group of a sweep takes (two runs of 32)
constexpr uint32_t kMaxComponents = 1024; // graphs in one batched handle

// Tier of an in-degree in the full/dense sweep order: 0 = one thread (<= lo), 1 = an
// 8-lane group (<= max(lo, gmax), gmax <= kGroupMax), 2 = chunks of `chunk` edges taken by
// whole warps (chunk <= kChunk).  gmax and chunk are tuning parameters of a handle.
__host__ __device__ inline int sweep_tier(uint32_t d, uint32_t lo, uint32_t gmax) {
  return d <= lo ? 0 : (d <= (lo > gmax ? lo : gmax) ? 1 : 2);
}

// ----------------------------------------------------------------- device helpers ---

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add_u32(uint32_t *p, uint32_t v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Kernel-launch accounting (pr_kernel_launches); bumped after every launch.
void count_launch();
void count_launches(unsigned long long k);
// Host-side fault injection (pr_inject_alloc_failure): true if this allocation must fail.
bool alloc_fault();

// ------------------------------------------------------------- rank storage ---
// Ranks R, cached contributions C[u] = alpha R[u] / |out(u)| and the per-vertex factor A
// that turns a rank into a contribution.
//
// 64-bit mode (PR_F64) computes in exact 64-bit fixed point with 62 fractional bits:
// R and C are int64 counts of 2^-62 (about 2.2e-19), A = alpha / |out(u)| as an unsigned
// 64-bit fraction, and C = round(R * A / 2^64) with one 64x64 -> 128-bit multiply.  Ranks
// enter and leave the library as IEEE doubles.  Why: GB300 issues FP64 arithmetic at a
// small fraction of its integer rate, and an FP64 add per gathered edge (plus a few FP64
// operations per vertex) bounded the sweep far below HBM bandwidth.  Every quantity the
// method compares is absolute (L-inf change <= tau, rank change > tau_f), so a fixed
// absolute resolution of 2^-62 serves it exactly: in-edge sums, L-inf maxima and the
// dead-end mass are exact integer operations, and each contribution is rounded once.
// All ranks are below 1 and every in-sum is at most its vertex's rank, so no value
// reaches 2^62.
// FP32 mode (PR_F32) keeps R, C and A in float.
template <bool F32>
struct Store;

template <>
struct Store<false> {
  using R = long long;
  using C = long long;
  using A = unsigned long long;
  static constexpr double kOne = 4611686018427387904.0;   // 2^62
  static constexpr double kFrac = 18446744073709551616.0;  // 2^64
  __device__ static A factor(double alpha, uint32_t d) { return d ? __double2ull_rn(alpha / (double)d * kFrac) : 0ull; }
  __device__ static C contrib(R r, A a) {
    const unsigned long long ur = (unsigned long long)r;
    const unsigned long long lo = ur * a, hi = __umul64hi(ur, a);
    return (long long)(hi + (lo >> 63));
  }
  __device__ static R from_double(double x) { return __double2ll_rn(x * kOne); }
  __device__ static double to_double(R r) { return (double)r * (1.0 / kOne); }
};

template <>
struct Store<true> {
  using R = float;
  using C = float;
  using A = float;
  __device__ static A factor(double alpha, uint32_t d) { return d ? (float)(alpha / (double)d) : 0.0f; }
  __device__ static C contrib(R r, A a) { return r * a; }
  __device__ static R from_double(double x) { return (float)x; }
  __device__ static double to_double(R r) { return (double)r; }
};

// ------------------------------------------------------------------- structures ---

// One adjacency (in- or out-edges) in slack-row form.
struct Adj {
  uint2 *rd = nullptr;      // [n] {start, len}
  uint32_t *cap = nullptr;  // [n] slots owned by the row (multiple of 4)
  uint32_t *col = nullptr;  // [col_cap]
  uint64_t col_cap = 0;     // words allocated for col
  uint64_t used = 0;        // words handed out (host mirror, refreshed after updates)
  uint64_t garbage = 0;     // words of rows abandoned by moves (host mirror)
};

// Device control block of the rank kernel; zeroed before every launch.
struct RankCtl {
  uint32_t bar;                                   // grid barrier arrivals (monotonic)
  uint32_t err;                                   // nonzero: a bounded wait gave up
  uint32_t err_where;
  uint32_t iterations;
  uint32_t converged;
  uint32_t full_from;                             // iteration from which all of V is affected (+1; 0 = never)
  uint32_t status;                                // split calls: what the last launch left to do
  uint32_t next_it;                               // split calls: iteration the next launch starts with
  uint32_t final_cnt[3];                          // affected-list lengths at the end (Dynamic Frontier)
  uint32_t pad;
  unsigned long long last_key;                    // L-inf change of the last iteration (see Num<>::key)
  double D_final;                                 // dead-end mass of the final ranks (FP32 mode)
  long long D_final_n;                            // the same in 2^-62 units (64-bit mode)
  unsigned long long dR_bits[kMaxIterLimit + 1];  // per-iteration L-inf (bits of a non-negative double)
  uint32_t tail[kMaxIterLimit + 2][4];            // per-iteration appends per bin ([0] = initial marks)
  uint32_t blk_next[kMaxIterLimit + 1];           // dynamic index into the block bin
  uint32_t cmp[kMaxIterLimit + 1][4];             // affected items per tier after a dense compaction
  unsigned long long hubq[kMaxIterLimit + 2];     // per slot: queued long out-rows << 32 | their chunks
  unsigned long long vproc, eproc, expv, expe, appended;
  uint32_t save_cnt[3], save_cmp[3], save_cmp_total;  // split calls: lists and compaction at the handoff
  uint32_t xcnt;                                      // entries of the expansion list (cursor)
  uint32_t xit[kMaxIterLimit + 2];                    // entries appended for each slot: read after the
                                                      // barrier, when no block can append to that slot
  uint32_t xneed[kMaxIterLimit + 2];                  // continuation: a recorded expansion would mark
  // per-iteration sweep launches (sweep.cu): what one launch leaves for the next
  uint32_t ticket;        // blocks of the current sweep launch that have finished
  uint32_t it_cur;        // iteration the next sweep launch computes
  uint32_t sw_all[3];     // sweep items per tier (all vertices)
  uint32_t sw_off[2];     // first item of tiers 1 and 2 (in the item and compacted arrays)
  uint32_t m_cur;         // stored edges (in-edges of all vertices)
  uint32_t dmode;         // dense Dynamic Frontier: 1 = every item swept with the stamp check, 0 = compacted items
  uint32_t pull_check;    // this iteration pulls marks from the previous iteration's changes
  uint32_t erec;          // this iteration records per-vertex change flags (the next may pull)
  uint32_t push_items;    // pushed marks append their sweep items to the compacted items
  uint32_t push_lo, push_n;   // the prologue pushes the out-rows of these expansion-list entries
  uint32_t compact_now;   // the prologue recompacts the affected items
  uint32_t dexpand;       // record first expansions (0 for Dynamic Traversal after its search)
  uint32_t xdone;         // expansion-list entries pushed or skipped
  uint32_t dcnt[3];       // affected-list lengths committed before the current iteration
  uint32_t cmp_cur[3];    // compacted items per tier, items of later marks appended
  uint32_t cmp_total;     // affected vertices when the compacted items were last rebuilt
  uint32_t app_since;     // vertices whose items were appended since then
  unsigned long long cmp_edges;  // in-edges of the vertices with compacted items (appended ones included)
  uint32_t kind_cur;      // trace kind of the current iteration
  uint32_t launches;      // sweep and prologue launches the device-side loop made
  uint32_t xcap;          // expansion-list entries this iteration writes at most (more: it only counts)
  uint32_t x_long;        // a compacted iteration listed a vertex with an out-row longer than kInlineOut
  uint32_t jtotal;        // vertices that joined by pulls (not in the lists)
  uint32_t dense_ran;     // the per-iteration loop ran: its writeback listed the affected set
  uint32_t aff_total;     // affected vertices listed by that writeback (list 0)
  uint32_t pull_all;      // the pull kernel also pulls tier-0/1 rows (the marks after the last iteration)
  unsigned long long bar_limit_ns;  // grid-barrier wait limit (0 = the default)
  uint32_t fin_only;      // a marking launch handed off only for the marks of its last iteration
  unsigned long long eprev;  // edges processed before the current iteration
  // trace (written by block 0): %globaltimer at kernel start, after phase 0 and after each
  // iteration's barrier; affected vertices at the start of each iteration; iteration kind
  unsigned long long t_ns[kMaxIterLimit + 2];
  uint32_t it_aff[kMaxIterLimit + 1];
  uint8_t it_kind[kMaxIterLimit + 1];  // 0 sparse, 1 dense (reused items), 2 dense (compacted), 3 full
};

// Per-block Neumaier partials of the dead-end mass, double-buffered by iteration parity.
struct DeadPart {
  double s, c;
};

// Scratch of a batch update.
struct ApplyScratch {
  uint64_t cap = 0;             // capacity in pairs
  uint32_t *pairs = nullptr;    // 4 * cap: del_src, del_dst, ins_src, ins_dst
  uint64_t *kd = nullptr, *tmp = nullptr, *tmp2 = nullptr;  // keys [cap] each
  uint64_t *chg = nullptr, *chg_t = nullptr;   // tagged change lists [2 cap]
  uint32_t *flags = nullptr, *pos = nullptr;   // [2 cap + 1]
  uint32_t *seg = nullptr;                      // segment starts [2 cap + 1]
  uint32_t *tagpref = nullptr;                  // [2 cap + 1]
  uint32_t *radix_hist = nullptr;               // radix histogram scratch
  uint64_t radix_hist_cap = 0;
  uint32_t *scan_tmp = nullptr;                 // scan block sums
  uint64_t scan_tmp_cap = 0;
  uint32_t *vals = nullptr, *vals2 = nullptr;   // (place << 1) | is_insertion [cap], sorted with the keys
  uint32_t *boff = nullptr;                     // batch offsets of a sequence [2 (boff_cap + 1)]
  int32_t boff_cap = 0;
};

// Device-side counters of a batch update (one struct, read back once).
struct ApplyCtl {
  uint32_t bad_id;
  uint32_t n_eff;        // effective changes (deletions + insertions)
  uint32_t n_seg_out, n_seg_in;
  unsigned long long reloc_out, reloc_in;   // words needed by rows that must move
  unsigned long long tail_out, tail_in;     // running allocation cursors (device)
  unsigned long long garbage_out, garbage_in;
  uint32_t n_pend_src, n_pend_tgt;          // pending marks after this update
  uint32_t pend_overflow;
  uint32_t dead_changed;
  uint32_t n_eff_del;                       // effective deletions among n_eff
  uint32_t overflow;                        // a merge found no room (graph left unchanged rows)
  uint32_t bins_changed;                    // an in-degree crossed a bin threshold
  uint32_t bad_comp;                        // a pair joins two graphs of a batched handle
  unsigned long long big_cursor;            // global scratch cursor for long rows
  uint32_t n_long;                          // rows left by the merge for its long-row pass
};

// ------------------------------------------------------------------- primitives ---
// All run on `st`; counts are host values.  Implemented in prim.cu.

// Exclusive scan of n uint32 values (out may alias in); returns nothing; tmp sized by
// scan_tmp_words(n).
size_t scan_tmp_words(uint64_t n);
void exclusive_scan_u32(const uint32_t *in, uint32_t *out, uint64_t n, uint32_t *tmp, cudaStream_t st);

// Sort n 64-bit keys on their low `bits` bits (stable LSD radix; one block when
// n <= kSmallSort).  keys and alt are both n long; the result is returned (one of them).
size_t radix_hist_words(uint64_t n);
uint64_t *sort_u64(uint64_t *keys, uint64_t *alt, uint64_t n, int bits, uint32_t *hist,
                   uint32_t *scan_tmp, cudaStream_t st);

// Stable sort of n (key, value) pairs by the key's low `bits` bits; *keys / *vals point at
// the result afterwards (the inputs or the alternates).
void sort_u64_kv(uint64_t **keys, uint32_t **vals, uint64_t *alt_k, uint32_t *alt_v, uint64_t n, int bits,
                 uint32_t *hist, uint32_t *scan_tmp, cudaStream_t st);

int bits_for(uint32_t n);  // bits needed for ids in [0, n), at least 1

}  // namespace prdf

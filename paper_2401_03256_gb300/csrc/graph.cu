// graph.cu - device graph store: build from pairs, batch update, repack, export.
//
// Section 3.2 of the paper defines a batch update as E^t = (E^{t-1} \ D) U I with
// effective deletions Delta^- = E^{t-1} \ E^t and insertions Delta^+ = E^t \ E^{t-1};
// Section 3.1 / 5.1.4 add a self-loop to every vertex (kept fixed across updates).
//
// Update pipeline (all on the handle's stream):
//   keys (u << b | v) of the requested pairs in sequence order -> stable sort -> the last
//   request on each edge decides its state, and the edges whose state changes are the
//   effective changes (self pairs, duplicates, deletions of absent edges, deletions that
//   are re-inserted and insertions of present edges drop out) -> tagged change list in
//   (u, v) order and a transposed copy sorted by (v, u) -> segments = touched rows -> one block
//   per touched row merges the row with its changes, in place if the row's slots
//   suffice, else into freshly allocated tail slots.  The out-row merge also refreshes
//   the row's contribution alpha R[u] / |out(u)| and records the pending marks
//   (sources and deleted targets) for the next Dynamic Frontier call.
#include <algorithm>
#include <vector>

#include "prdf_graph.cuh"

namespace prdf {

#define CK(call)                                            \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(g, e_, #call);  \
  } while (0)

pr_status cuda_fail(Graph *g, cudaError_t e, const char *what) {
  g->err = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? PR_ERR_OUT_OF_MEMORY : PR_ERR_CUDA;
}

template <class T>
static cudaError_t dalloc(T **p, uint64_t count) {
  *p = nullptr;
  if (alloc_fault()) return cudaErrorMemoryAllocation;
  return cudaMalloc((void **)p, sizeof(T) * (count ? count : 1));
}

static inline unsigned grid_for(uint64_t n, int threads = 256) {
  uint64_t g = (n + threads - 1) / threads;
  return (unsigned)std::max<uint64_t>(1, g);
}

constexpr int kMergeThreads = 256;
constexpr int kMergeThreadsLong = 1024;
constexpr uint32_t kSmemRow = 2048;   // rows up to this length are staged in shared memory
#ifndef PRDF_LONG_ROW
#define PRDF_LONG_ROW 8192
#endif
constexpr uint32_t kLongRow = PRDF_LONG_ROW;  // longer rows are merged by blocks of kMergeThreadsLong

// ------------------------------------------------------------------- kernels ----

__global__ void k_validate_pairs(const uint32_t *src, const uint32_t *dst, uint64_t m, uint32_t n, uint32_t *bad) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m && (src[i] >= n || dst[i] >= n)) atomicOr(bad, 1u);
}

// Keys (u << b | v) of the input pairs (self pairs become the sentinel), followed by the
// n self-loop keys when self_loops is set.
__global__ void k_make_keys(const uint32_t *src, const uint32_t *dst, uint64_t m_in, uint32_t n, int b,
                            int self_loops, uint64_t *keys) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m_in) {
    uint64_t u = src[i], v = dst[i];
    keys[i] = u == v ? kSentinel : ((u << b) | v);
  } else if (self_loops && i < m_in + n) {
    uint64_t v = i - m_in;
    keys[i] = (v << b) | v;
  }
}

__device__ __forceinline__ uint32_t unique_flag(const uint64_t *keys, uint64_t i) {
  uint64_t k = keys[i];
  return (k != kSentinel && (i == 0 || keys[i - 1] != k)) ? 1u : 0u;
}

__global__ void k_unique_flags(const uint64_t *keys, uint64_t m, uint32_t *flags) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) flags[i] = unique_flag(keys, i);
}

__global__ void k_compact_unique(const uint64_t *keys, const uint32_t *pos, uint64_t m, uint64_t *out,
                                 uint32_t *count) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  uint32_t f = unique_flag(keys, i);
  if (f) out[pos[i]] = keys[i];
  if (i == m - 1) *count = pos[i] + f;
}

__global__ void k_transpose_keys(const uint64_t *keys, uint64_t m, int b, uint64_t *out) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  uint64_t k = keys[i], mask = (1ull << b) - 1;
  out[i] = ((k & mask) << b) | (k >> b);
}

// off[r] = index of the first key of row r (rows are key >> b); off[n] = m.
__global__ void k_row_bounds(const uint64_t *keys, uint64_t m, int b, uint32_t n, uint32_t *off) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > m) return;
  int64_t prev = i == 0 ? -1 : (int64_t)(keys[i - 1] >> b);
  int64_t cur = i == m ? (int64_t)n : (int64_t)(keys[i] >> b);
  for (int64_t r = prev + 1; r <= cur; r++) off[r] = (uint32_t)i;
}

__global__ void k_row_caps(const uint32_t *off, uint32_t n, uint32_t *cap) {
  uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) cap[v] = slack_cap(off[v + 1] - off[v]);
}

__global__ void k_row_desc(const uint32_t *start, const uint32_t *off, uint32_t n, uint2 *rd) {
  uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) rd[v] = make_uint2(start[v], off[v + 1] - off[v]);
}

__global__ void k_scatter_cols(const uint64_t *keys, uint64_t m, int b, const uint32_t *off, const uint2 *rd,
                               uint32_t *col) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  uint64_t k = keys[i];
  uint32_t r = (uint32_t)(k >> b);
  col[rd[r].x + (uint32_t)(i - off[r])] = (uint32_t)(k & ((1ull << b) - 1));
}

template <bool F32>
__global__ void k_init_rank(const uint2 *out_rd, uint32_t n, double alpha, typename Store<F32>::A *adeg,
                            typename Store<F32>::R *R0, typename Store<F32>::R *R1, typename Store<F32>::C *C0,
                            typename Store<F32>::C *C1) {
  using S = Store<F32>;
  uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  typename S::A a = S::factor(alpha, out_rd[v].y);
  typename S::R r = S::from_double(1.0 / (double)n);
  typename S::C c = S::contrib(r, a);
  adeg[v] = a;
  R0[v] = r;
  R1[v] = r;
  C0[v] = c;
  C1[v] = c;
}

// ---- batch update ----

// Chunk items of the tier-2 rows; chunk c of a row covers edges [c chunk, (c+1) chunk).
__device__ __forceinline__ uint4 chunk_item(uint32_t v, uint2 d, uint32_t c, uint32_t nch, uint32_t number,
                                            uint32_t chunk) {
  uint32_t len = min(chunk, d.y - c * chunk);
  return make_uint4(v, d.x + c * chunk, len | (c << 10) | (nch > 1 ? 0x80000000u : 0u), number);
}


__device__ __forceinline__ bool row_has(const uint2 *rd, const uint32_t *col, uint32_t u, uint32_t v) {
  uint2 d = rd[u];
  const uint32_t *c = col + d.x;
  uint32_t lo = 0, hi = d.y;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (c[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo < d.y && c[lo] == v;
}

__device__ __forceinline__ bool sorted_has(const uint64_t *a, uint64_t n, uint64_t x) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    uint64_t mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo < n && a[lo] == x;
}

// Batch k of a sequence holding op x of one kind: the last k with off[k] <= x.
__device__ __forceinline__ uint32_t batch_of(const uint32_t *off, int nb, uint64_t x) {
  uint32_t lo = 0, hi = (uint32_t)nb;  // off[0] = 0 <= x
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (off[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

// Keys (u << b | v) of a sequence of batches, each request written at its place in the
// order D_0, I_0, D_1, I_1, ... (deletions before insertions inside a batch, Section 3.2),
// with the payload (place << 1) | is_insertion.  off = [del offsets (nb + 1), ins offsets
// (nb + 1)], or null for a single batch.
__global__ void k_seq_keys(const uint32_t *ds, const uint32_t *dd, uint64_t nd, const uint32_t *is,
                           const uint32_t *id, uint64_t ni, int nb, const uint32_t *off, uint32_t n, int b,
                           uint64_t *keys, uint32_t *vals, const uint16_t *comp, const uint32_t *inv,
                           ApplyCtl *actl) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nd + ni) return;
  uint64_t u, v, at;
  uint32_t kind;
  if (i < nd) {
    u = ds[i];
    v = dd[i];
    kind = 0;
    at = off ? off[nb + 1 + batch_of(off, nb, i)] + i : i;
  } else {
    const uint64_t j = i - nd;
    u = is[j];
    v = id[j];
    kind = 1;
    at = off ? off[batch_of(off + nb + 1, nb, j) + 1] + j : nd + j;
  }
  uint64_t key;
  if (u >= n || v >= n) {
    atomicOr(&actl->bad_id, 1u);
    key = kSentinel;
  } else if (comp && comp[u] != comp[v]) {
    atomicOr(&actl->bad_comp, 1u);
    key = kSentinel;
  } else {
    if (inv) {  // the handle's internal numbering
      u = inv[u];
      v = inv[v];
    }
    key = u == v ? kSentinel : ((u << b) | v);
  }
  keys[at] = key;
  vals[at] = (uint32_t)(at << 1) | kind;
}

// After the stable sort every key's requests sit together in sequence order, so the last
// one fixes the edge's final state; flags[i] = 1 where that state differs from the graph's
// (an effective deletion or insertion).  Self pairs and repeated requests never count.
__global__ void k_last_op(const uint64_t *keys, const uint32_t *vals, uint64_t N, const uint2 *rd,
                          const uint32_t *col, int b, uint32_t *flags) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const uint64_t k = keys[i];
  uint32_t keep = 0;
  if (k != kSentinel && (i + 1 == N || keys[i + 1] != k)) {
    const bool fin = vals[i] & 1u;
    const bool was = row_has(rd, col, (uint32_t)(k >> b), (uint32_t)(k & ((1ull << b) - 1)));
    keep = fin != was;
  }
  flags[i] = keep;
}

// Tagged change keys: (key << 1) | is_insertion, in row-major (u, v) order and a
// transposed (v, u) copy.
__global__ void k_emit_changes(const uint64_t *keys, const uint32_t *vals, uint64_t N, const uint32_t *flags,
                               const uint32_t *pos, int b, uint64_t *chg, uint64_t *chg_t, ApplyCtl *actl) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (flags[i]) {
    const uint64_t k = keys[i];
    const uint64_t tag = vals[i] & 1u;
    const uint64_t mask = (1ull << b) - 1;
    const uint64_t kt = ((k & mask) << b) | (k >> b);
    chg[pos[i]] = (k << 1) | tag;
    chg_t[pos[i]] = (kt << 1) | tag;
    if (!tag) atomicAdd(&actl->n_eff_del, 1u);
  }
  if (i == N - 1) actl->n_eff = pos[i] + flags[i];
}

__device__ __forceinline__ uint32_t chg_row(uint64_t c, int b) { return (uint32_t)((c >> 1) >> b); }
__device__ __forceinline__ uint32_t chg_col(uint64_t c, int b) { return (uint32_t)((c >> 1) & ((1ull << b) - 1)); }

// flags[j] = start of a row segment; tags[j] = is_insertion; tags[K] = 0.
__global__ void k_seg_flags(const uint64_t *chg, uint32_t K, int b, uint32_t *flags, uint32_t *tags) {
  uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < K) {
    flags[j] = (j == 0 || chg_row(chg[j], b) != chg_row(chg[j - 1], b)) ? 1u : 0u;
    tags[j] = (uint32_t)(chg[j] & 1);
  } else if (j == K) {
    tags[j] = 0;
  }
}

__global__ void k_seg_emit(const uint32_t *flags, const uint32_t *pos, uint32_t K, uint32_t *seg, uint32_t *nseg) {
  uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= K) return;
  if (flags[j]) seg[pos[j]] = j;
  if (j == K - 1) {
    uint32_t c = pos[j] + flags[j];
    seg[c] = K;
    *nseg = c;
  }
}

// Words the moved rows need, and the long rows' staging words.
__global__ void k_plan(const uint2 *rd, const uint32_t *cap, const uint64_t *chg, uint32_t K, int b,
                       const uint32_t *seg, const uint32_t *nseg, const uint32_t *tagpref,
                       unsigned long long *reloc, unsigned long long *big_need) {
  uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= *nseg) return;
  uint32_t s0 = seg[s], e = seg[s + 1];
  uint32_t r = chg_row(chg[s0], b);
  uint32_t nI = tagpref[e] - tagpref[s0], nD = (e - s0) - nI;
  uint32_t len = rd[r].y;
  uint32_t new_len = len - nD + nI;
  if (new_len > cap[r]) atomicAdd(reloc, (unsigned long long)move_cap(new_len));
  if (len > kSmemRow) atomicAdd(big_need, (unsigned long long)len);
}

// Extra work done by the merge of a row.  Out-rows (source u): contribution refresh and
// pending marks.  In-rows: note an in-degree that crosses a bin threshold.
template <bool F32>
struct RowHook {
  bool is_out;
  double alpha;
  typename Store<F32>::A *adeg;
  typename Store<F32>::R *R0;
  typename Store<F32>::C *C0, *C1;
  uint32_t *pend_src, *pend_tgt;
  uint32_t pend_cap;
  uint32_t bin_lo, bin_hi;
  uint32_t gmax, chunk;       // sweep tiers of the handle (sweep_tier)
  uint4 *items;               // in-rows: sweep items to patch (tier and chunk count unchanged)
  const uint32_t *item_pos;
};

__device__ __forceinline__ int degree_bin(uint32_t d, uint32_t lo, uint32_t hi) {
  return d <= lo ? 0 : (d <= hi ? 1 : 2);
}

// Merges one touched row (segment s of the sorted changes) with its changes; called by a
// whole block.
template <bool F32, int THREADS>
__device__ void merge_row(uint32_t s, uint2 *rd, uint32_t *cap, uint32_t *col, const uint64_t *chg, int b,
                          const uint32_t *seg, const uint32_t *tagpref, unsigned long long *tail,
                          unsigned long long *garbage, uint32_t *big, unsigned long long *big_cursor,
                          uint64_t col_cap, uint64_t big_cap, ApplyCtl *actl, const RowHook<F32> &hook) {
  constexpr int kMergeThreads = THREADS;
  __shared__ uint32_t srow[kSmemRow];
  __shared__ uint32_t s_dest, s_big;
  const uint32_t tid = threadIdx.x;
  const uint32_t s0 = seg[s], e = seg[s + 1];
  const uint32_t r = chg_row(chg[s0], b);
  const uint2 d = rd[r];
  const uint32_t len = d.y, cap_r = cap[r];
  const uint32_t nI = tagpref[e] - tagpref[s0], nD = (e - s0) - nI;
  const uint32_t new_len = len - nD + nI;
  const bool moves = new_len > cap_r;
  uint32_t *src_row = srow;
  __shared__ int s_ok;
  if (tid == 0) {
    unsigned long long dest = moves ? atomicAdd(tail, (unsigned long long)move_cap(new_len)) : d.x;
    unsigned long long bg = len > kSmemRow ? atomicAdd(big_cursor, (unsigned long long)len) : 0ull;
    s_ok = (!moves || dest + move_cap(new_len) <= col_cap) && (len <= kSmemRow || bg + len <= big_cap);
    if (!s_ok) atomicOr(&actl->overflow, 1u);
    s_dest = (uint32_t)dest;
    s_big = (uint32_t)bg;
  }
  __syncthreads();
  if (!s_ok) return;  // no room: the row is left as it was and the host reports the failure
  if (len > kSmemRow) src_row = big + s_big;
  for (uint32_t j = tid; j < len; j += kMergeThreads) src_row[j] = col[d.x + j];
  __syncthreads();
  uint32_t *dst = col + s_dest;
  // A thread's entries ascend, so the first change with column >= x lies at or after the
  // one found for its previous entry: a galloping search from there (a hub row's entries
  // are each a few changes apart, not a whole binary search over them).
  uint32_t lo_prev = s0;
  for (uint32_t j = tid; j < len; j += kMergeThreads) {
    uint32_t x = src_row[j];
    uint32_t lo = lo_prev, hi = lo_prev, step = 1;  // changes before lo have columns < x
    while (hi < e && chg_col(chg[hi], b) < x) {
      lo = hi + 1;
      hi = e - hi > step ? hi + step : e;
      step <<= 1;
    }
    while (lo < hi) {  // first change with column >= x, in [lo, hi]
      uint32_t mid = (lo + hi) >> 1;
      if (chg_col(chg[mid], b) < x) lo = mid + 1; else hi = mid;
    }
    lo_prev = lo;
    if (lo < e && chg_col(chg[lo], b) == x) continue;  // deleted
    uint32_t ib = tagpref[lo] - tagpref[s0];
    uint32_t db = (lo - s0) - ib;
    dst[j - db + ib] = x;
  }
  for (uint32_t q = s0 + tid; q < e; q += kMergeThreads) {
    uint64_t c = chg[q];
    if (!(c & 1)) continue;
    uint32_t y = chg_col(c, b);
    uint32_t lo = 0, hi = len;  // old entries below y
    while (lo < hi) {
      uint32_t mid = (lo + hi) >> 1;
      if (src_row[mid] < y) lo = mid + 1; else hi = mid;
    }
    uint32_t ib = tagpref[q] - tagpref[s0];
    uint32_t db = (q - s0) - ib;
    dst[lo - db + ib] = y;
  }
  if (hook.is_out) {
    for (uint32_t q = s0 + tid; q < e; q += kMergeThreads) {
      uint64_t c = chg[q];
      if (c & 1) continue;
      uint32_t p = atomicAdd(&actl->n_pend_tgt, 1u);
      if (p < hook.pend_cap) hook.pend_tgt[p] = chg_col(c, b);
    }
  }
  __syncthreads();
  if (tid == 0) {
    rd[r] = make_uint2(s_dest, new_len);
    if (moves) {
      cap[r] = move_cap(new_len);
      atomicAdd(garbage, (unsigned long long)cap_r);
    }
    if (!hook.is_out && (sweep_tier(len, hook.bin_lo, hook.gmax) != sweep_tier(new_len, hook.bin_lo, hook.gmax) ||
                         (sweep_tier(new_len, hook.bin_lo, hook.gmax) == 2 &&
                          (len + hook.chunk - 1) / hook.chunk != (new_len + hook.chunk - 1) / hook.chunk))) {
      actl->bins_changed = 1;
      s_ok = 0;  // the sweep items are rebuilt after this update; nothing to patch
    }
    if (hook.is_out) {
      using S = Store<F32>;
      typename S::A a = S::factor(hook.alpha, new_len);
      hook.adeg[r] = a;
      typename S::C c = S::contrib(hook.R0[r], a);
      hook.C0[r] = c;
      hook.C1[r] = c;
      if ((len == 0) != (new_len == 0)) actl->dead_changed = 1;
      uint32_t p = atomicAdd(&actl->n_pend_src, 1u);
      if (p < hook.pend_cap) hook.pend_src[p] = r;
    }
  }
  if (!hook.is_out) {
    // keep the sweep items of this in-row current (start and length)
    __syncthreads();
    if (s_ok) {
      const uint2 nd = make_uint2(s_dest, new_len);
      const uint32_t pos = hook.item_pos[r];
      if (sweep_tier(new_len, hook.bin_lo, hook.gmax) < 2) {
        if (tid == 0) hook.items[pos] = make_uint4(r, nd.x, nd.y, 0u);
      } else {
        const uint32_t nch = (new_len + hook.chunk - 1) / hook.chunk;
        const uint32_t number0 = hook.items[pos].w;
        for (uint32_t c = tid; c < nch; c += kMergeThreads)
          hook.items[pos + c] = chunk_item(r, nd, c, nch, number0 + c, hook.chunk);
      }
    }
  }
}

// One block per touched row of at most kLongRow entries; the longer rows are listed (their
// segments in long_seg) for k_merge_long, whose blocks of kMergeThreadsLong take them in
// turn: a hub row's entries are four times as many threads' work, and only as many blocks
// as the GPU holds are launched for them.
template <bool F32>
__global__ void __launch_bounds__(kMergeThreads) k_merge(uint2 *rd, uint32_t *cap, uint32_t *col, const uint64_t *chg,
                                                         int b, const uint32_t *seg, const uint32_t *nseg,
                                                         const uint32_t *tagpref, unsigned long long *tail,
                                                         unsigned long long *garbage, uint32_t *big,
                                                         unsigned long long *big_cursor, uint64_t col_cap,
                                                         uint64_t big_cap, ApplyCtl *actl, RowHook<F32> hook,
                                                         uint32_t *long_seg) {
  const uint32_t s = blockIdx.x;
  if (s >= *nseg) return;
  if (rd[chg_row(chg[seg[s]], b)].y > kLongRow) {
    if (threadIdx.x == 0) long_seg[atomicAdd(&actl->n_long, 1u)] = s;
    return;
  }
  merge_row<F32, kMergeThreads>(s, rd, cap, col, chg, b, seg, tagpref, tail, garbage, big, big_cursor, col_cap,
                                big_cap, actl, hook);
}

template <bool F32>
__global__ void __launch_bounds__(kMergeThreadsLong) k_merge_long(uint2 *rd, uint32_t *cap, uint32_t *col,
                                                                  const uint64_t *chg, int b, const uint32_t *seg,
                                                                  const uint32_t *tagpref, unsigned long long *tail,
                                                                  unsigned long long *garbage, uint32_t *big,
                                                                  unsigned long long *big_cursor, uint64_t col_cap,
                                                                  uint64_t big_cap, ApplyCtl *actl,
                                                                  RowHook<F32> hook, const uint32_t *long_seg) {
  const uint32_t n_long = *(volatile uint32_t *)&actl->n_long;
  for (uint32_t k = blockIdx.x; k < n_long; k += gridDim.x) {
    merge_row<F32, kMergeThreadsLong>(long_seg[k], rd, cap, col, chg, b, seg, tagpref, tail, garbage, big, big_cursor,
                                      col_cap, big_cap, actl, hook);
    __syncthreads();  // the block's shared staging is reused by its next row
  }
}

// ---- repack / export / bins ----

__global__ void k_len_caps(const uint2 *rd, uint32_t n, uint32_t *cap) {
  uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) cap[v] = slack_cap(rd[v].y);
}

// One warp per row: copies the row to new_col + start[v] and points rd at it.
__global__ void k_repack_rows(uint2 *rd, uint32_t n, const uint32_t *old_col, uint32_t *new_col,
                              const uint32_t *start) {
  uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint32_t lane = threadIdx.x & 31;
  if (w >= n) return;
  uint2 d = rd[w];
  uint32_t s = start[w];
  for (uint32_t j = lane; j < d.y; j += 32) new_col[s + j] = old_col[d.x + j];
  __syncwarp();
  if (lane == 0) rd[w] = make_uint2(s, d.y);
}

__global__ void k_row_len(const uint2 *rd, uint32_t n, uint32_t *len) {
  uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) len[v] = rd[v].y;
  else if (v == n) len[v] = 0;
}

__global__ void k_pack_rows(const uint2 *rd, uint32_t n, const uint32_t *col, const uint32_t *off, uint32_t *packed) {
  uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint32_t lane = threadIdx.x & 31;
  if (w >= n) return;
  uint2 d = rd[w];
  uint32_t o = off[w];
  for (uint32_t j = lane; j < d.y; j += 32) packed[o + j] = col[d.x + j];
}

__global__ void k_dead_flags(const uint2 *rd, uint32_t n, uint32_t *flags) {
  uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) flags[v] = rd[v].y == 0;
}

// Stable compaction of the ids whose flag is set; count = total.
// Sweep-item rebuild in two passes over the vertices (tile of kIdentTile per block): the
// first counts each tile's vertices per tier and the chunk items of its tier-2 rows; after
// one exclusive scan of those counts (tier 0, 1, 2 tiles back to back, then the chunk
// counts), the second writes every vertex's item(s) at its place, in ascending vertex order
// within each tier.
constexpr uint32_t kIdentTile = 4096;

__global__ void k_tier_counts(const uint2 *rd, uint32_t n, uint32_t lo, uint32_t gmax, uint32_t chunk,
                              uint32_t nblk, uint32_t *bcnt, uint32_t *over) {
  __shared__ uint32_t s[4][8];
  const uint32_t tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint32_t base = blockIdx.x * kIdentTile;
  uint32_t c[4] = {0u, 0u, 0u, 0u};
  for (uint32_t k = tid; k < kIdentTile; k += 256) {
    const uint32_t v = base + k;
    if (v < n) {
      const uint32_t d = rd[v].y;
      const int t = sweep_tier(d, lo, gmax);
      c[t]++;
      if (t == 2) {
        const uint32_t ch = (d + chunk - 1) / chunk;
        c[3] += ch;
        if (ch > (1u << 21)) *over = 1u;  // a chunk's index within its row has 21 bits
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 4; j++) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c[j] += __shfl_xor_sync(0xffffffffu, c[j], o);
    if (lane == 0) s[j][w] = c[j];
  }
  __syncthreads();
  if (tid < 4) {
    uint32_t t = 0;
    for (int k = 0; k < 8; k++) t += s[tid][k];
    // tiers 0-2 back to back, a zero, the chunk counts, a zero
    bcnt[tid < 3 ? tid * nblk + blockIdx.x : 3 * nblk + 1 + blockIdx.x] = t;
  }
  if (blockIdx.x == 0 && tid == 0) {
    bcnt[3 * nblk] = 0u;
    bcnt[4 * nblk + 1] = 0u;
  }
}

__global__ void k_items_write(const uint2 *rd, uint32_t n, uint32_t lo, uint32_t gmax, uint32_t chunk,
                              uint32_t nblk, const uint32_t *bpos, uint4 *items, uint32_t *item_pos) {
  __shared__ uint32_t s[4][8];
  __shared__ uint32_t s_at[4];
  const uint32_t tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint32_t base = blockIdx.x * kIdentTile;
  // item positions of this tile's first vertex of tiers 0 and 1, and of its first chunk item
  // (the chunk items follow the items of tiers 0 and 1, bpos[2 * nblk] of them)
  const uint32_t c01 = bpos[2 * nblk];
  if (tid < 3) s_at[tid] = bpos[tid * nblk + blockIdx.x];
  if (tid == 3) s_at[3] = c01 + bpos[3 * nblk + 1 + blockIdx.x] - bpos[3 * nblk + 1];
  __syncthreads();
  for (uint32_t r0 = 0; r0 < kIdentTile; r0 += 256) {
    const uint32_t v = base + r0 + tid;
    uint2 d = make_uint2(0u, 0u);
    int t = -1;
    uint32_t ch = 0;
    if (v < n) {
      d = rd[v];
      t = sweep_tier(d.y, lo, gmax);
      if (t == 2) ch = (d.y + chunk - 1) / chunk;
    }
    // rank within the warp per tier, chunk prefix within the warp
    uint32_t m[3], incl = ch;
#pragma unroll
    for (int j = 0; j < 3; j++) m[j] = __ballot_sync(0xffffffffu, t == j);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (uint32_t)o) incl += y;
    }
    if (lane == 31) s[3][w] = incl;
    if (lane < 3) s[lane][w] = __popc(m[lane]);
    __syncthreads();
    uint32_t before[4] = {0u, 0u, 0u, 0u}, all[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int j = 0; j < 4; j++)
      for (int k = 0; k < 8; k++) {
        before[j] += k < (int)w ? s[j][k] : 0u;
        all[j] += s[j][k];
      }
    if (t >= 0 && t < 2) {
      const uint32_t pos = s_at[t] + before[t] + __popc(m[t] & ((1u << lane) - 1u));
      items[pos] = make_uint4(v, d.x, d.y, 0u);
      item_pos[v] = pos;
    } else if (t == 2) {
      const uint32_t first = s_at[3] + before[3] + incl - ch;  // index of the row's first chunk item
      const uint32_t number = first - c01;                     // its chunk number
      for (uint32_t c = 0; c < ch; c++) {
        const uint32_t len = min(chunk, d.y - c * chunk);
        items[first + c] = make_uint4(v, d.x + c * chunk, len | (c << 10) | (ch > 1 ? 0x80000000u : 0u), number + c);
      }
      item_pos[v] = first;
    }
    __syncthreads();
    if (tid < 4) s_at[tid] += all[tid];
    __syncthreads();
  }
}

__global__ void k_compact_ids(const uint32_t *flags, const uint32_t *pos, uint32_t n, uint32_t *out, uint32_t *count) {
  uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  if (flags[v]) out[pos[v]] = v;
  if (v == n - 1) *count = pos[v] + flags[v];
}

// ------------------------------------------------------------------ host side ---

static pr_status build_adj(Graph *g, const uint64_t *keys, uint64_t m, Adj &A, uint32_t *off, uint32_t *tmp,
                           uint32_t *scan_tmp) {
  const uint32_t n = g->n;
  cudaStream_t st = g->st;
  CK(dalloc(&A.rd, n));
  CK(dalloc(&A.cap, n));
  k_row_bounds<<<grid_for(m + 1), 256, 0, st>>>(keys, m, g->b, n, off); count_launch();
  k_row_caps<<<grid_for(n), 256, 0, st>>>(off, n, A.cap); count_launch();
  exclusive_scan_u32(A.cap, tmp, n, scan_tmp, st);
  uint32_t last[2];
  CK(cudaMemcpyAsync(&last[0], tmp + (n - 1), 4, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&last[1], A.cap + (n - 1), 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  uint64_t total = (uint64_t)last[0] + last[1];
  uint64_t reserve = std::max<uint64_t>(total / 4, 1024);
  reserve = (reserve + 3) & ~3ull;
  if (total + reserve > 0xFFFFFFFFull) {
    g->err = "graph too large: more than 2^32 - 1 column slots";
    return PR_ERR_CAPACITY;
  }
  A.col_cap = total + reserve;
  CK(dalloc(&A.col, A.col_cap));
  CK(cudaMemsetAsync(A.col, 0, sizeof(uint32_t) * A.col_cap, st));
  k_row_desc<<<grid_for(n), 256, 0, st>>>(tmp, off, n, A.rd); count_launch();
  k_scatter_cols<<<grid_for(m), 256, 0, st>>>(keys, m, g->b, off, A.rd, A.col); count_launch();
  A.used = total;
  A.garbage = 0;
  CK(cudaGetLastError());
  return PR_OK;
}

pr_status graph_build(Graph *g, uint64_t m_in, const uint32_t *src_d, const uint32_t *dst_d) {
  const uint32_t n = g->n;
  cudaStream_t st = g->st;
  g->b = bits_for(n);
  const bool sl = !g->teleport;
  const uint64_t mk = m_in + (sl ? n : 0);
  // validation before anything else
  uint32_t *flag = nullptr;
  CK(dalloc(&flag, 1));
  CK(cudaMemsetAsync(flag, 0, 4, st));
  if (m_in) {
    k_validate_pairs<<<grid_for(m_in), 256, 0, st>>>(src_d, dst_d, m_in, n, flag);
    count_launch();
  }
  uint32_t bad = 0;
  CK(cudaMemcpyAsync(&bad, flag, 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  cudaFree(flag);
  if (bad) {
    g->err = "vertex id out of range";
    return PR_ERR_VERTEX_RANGE;
  }
  if ((double)mk * 1.13 + 6.0 * n > 4.0e9) {
    g->err = "graph too large: more than 2^32 - 1 column slots";
    return PR_ERR_CAPACITY;
  }
  // scratch for the build
  uint64_t *keys = nullptr, *alt = nullptr;
  uint32_t *flags = nullptr, *pos = nullptr, *hist = nullptr, *stmp = nullptr, *cnt = nullptr;
  const uint64_t mk1 = std::max<uint64_t>(mk, 1);
  const uint64_t big = std::max<uint64_t>(mk1 + 1, (uint64_t)n + 1);
  pr_status rc = PR_OK;
  auto cleanup = [&]() {
    cudaFree(keys); cudaFree(alt); cudaFree(flags); cudaFree(pos); cudaFree(hist); cudaFree(stmp); cudaFree(cnt);
  };
  cudaError_t e = cudaSuccess;
  if ((e = dalloc(&keys, mk1)) != cudaSuccess || (e = dalloc(&alt, mk1)) != cudaSuccess ||
      (e = dalloc(&flags, big)) != cudaSuccess || (e = dalloc(&pos, big)) != cudaSuccess ||
      (e = dalloc(&hist, std::max(radix_hist_words(mk1), scan_tmp_words(big)) + 1)) != cudaSuccess ||
      (e = dalloc(&stmp, scan_tmp_words(std::max<uint64_t>(big, radix_hist_words(mk1))) + 1)) != cudaSuccess ||
      (e = dalloc(&cnt, 1)) != cudaSuccess) {
    cleanup();
    return cuda_fail(g, e, "graph build scratch");
  }
  do {
    if (mk) {
    k_make_keys<<<grid_for(mk), 256, 0, st>>>(src_d, dst_d, m_in, n, g->b, sl ? 1 : 0, keys);
    count_launch();
  }
    uint64_t *sorted = sort_u64(keys, alt, mk, 2 * g->b, hist, stmp, st);
    uint64_t *other = sorted == keys ? alt : keys;
    uint32_t m = 0;
    if (mk) {
      k_unique_flags<<<grid_for(mk), 256, 0, st>>>(sorted, mk, flags); count_launch();
      exclusive_scan_u32(flags, pos, mk, stmp, st);
      k_compact_unique<<<grid_for(mk), 256, 0, st>>>(sorted, pos, mk, other, cnt); count_launch();
      if ((e = cudaMemcpyAsync(&m, cnt, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
    }
    g->m = m;
    // out-adjacency from keys sorted by (u, v)
    rc = build_adj(g, other, m, g->out, flags, pos, stmp);
    if (rc != PR_OK) break;
    // in-adjacency from transposed keys sorted by (v, u)
    if (m) {
    k_transpose_keys<<<grid_for(m), 256, 0, st>>>(other, m, g->b, sorted);
    count_launch();
  }
    uint64_t *tsorted = sort_u64(sorted, other, m, 2 * g->b, hist, stmp, st);
    rc = build_adj(g, tsorted, m, g->in, flags, pos, stmp);
    if (rc != PR_OK) break;
    e = cudaStreamSynchronize(st);
  } while (0);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(g, e, "graph build");
  if (rc != PR_OK) return rc;

  // rank state
  const size_t es = g->f32 ? 4 : 8;
  for (int i = 0; i < 2; i++) {
    CK(cudaMalloc(&g->R[i], es * n));
    CK(cudaMalloc(&g->C[i], es * n));
  }
  CK(cudaMalloc(&g->adeg, es * n));
  const uint32_t words = (n + 31) / 32;
  CK(dalloc(&g->bitmap, words));
  CK(cudaMemsetAsync(g->bitmap, 0, 4ull * words, st));
  CK(dalloc(&g->xbits, words));
  CK(cudaMemsetAsync(g->xbits, 0, 4ull * words, st));
  CK(dalloc(&g->stamp, n));
  CK(cudaMemsetAsync(g->stamp, 0xFF, 2ull * n, st));
  CK(dalloc(&g->chunk_done, n));
  CK(cudaMemsetAsync(g->chunk_done, 0, 4ull * n, st));
  CK(dalloc(&g->item_pos, n));
  CK(dalloc(&g->hub_v, n));
  CK(dalloc(&g->hub_base, n));
  for (int i = 0; i < 3; i++) CK(dalloc(&g->list[i], n));
  CK(dalloc(&g->xlist, n));
  CK(dalloc(&g->dead, n));
  // (n + 8 words: also the sweep-item rebuild's 4 ceil(n / 4096) + 2 tile counts)
  CK(dalloc(&g->gen_tmp, (uint64_t)n + 8));
  CK(dalloc(&g->gen_tmp2, (uint64_t)n + 8));
  CK(dalloc(&g->scan_tmp, scan_tmp_words((uint64_t)n + 8) + 1));
  g->pend_cap = std::max<uint32_t>(1u << 16, std::min<uint32_t>(n, 1u << 22));
  CK(dalloc(&g->pend_src, g->pend_cap));
  CK(dalloc(&g->pend_tgt, g->pend_cap));
  CK(dalloc(&g->actl, 1));
  CK(cudaMallocHost((void **)&g->actl_h, sizeof(ApplyCtl)));
  if (g->f32) {
    using S = Store<true>;
    k_init_rank<true><<<grid_for(n), 256, 0, st>>>(g->out.rd, n, g->p.alpha, (S::A *)g->adeg, (S::R *)g->R[0],
                                                   (S::R *)g->R[1], (S::C *)g->C[0], (S::C *)g->C[1]);
  } else {
    using S = Store<false>;
    k_init_rank<false><<<grid_for(n), 256, 0, st>>>(g->out.rd, n, g->p.alpha, (S::A *)g->adeg, (S::R *)g->R[0],
                                                    (S::R *)g->R[1], (S::C *)g->C[0], (S::C *)g->C[1]);
  }
  count_launch();
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  g->ident_dirty = true;
  g->dead_dirty = true;
  return graph_refresh_ident(g);
}

pr_status apply_scratch(Graph *g, uint64_t N) {
  ApplyScratch &s = g->sc;
  if (N <= s.cap && s.pairs) return PR_OK;
  uint64_t cap = std::max<uint64_t>(N, 4096);
  uint32_t *boff = s.boff;
  const int32_t boff_cap = s.boff_cap;
  cudaFree(s.pairs); cudaFree(s.kd); cudaFree(s.vals); cudaFree(s.vals2); cudaFree(s.tmp); cudaFree(s.tmp2);
  cudaFree(s.chg); cudaFree(s.chg_t); cudaFree(s.flags); cudaFree(s.pos); cudaFree(s.seg);
  cudaFree(s.tagpref); cudaFree(s.radix_hist); cudaFree(s.scan_tmp);
  s = ApplyScratch{};
  s.boff = boff;
  s.boff_cap = boff_cap;
  CK(dalloc(&s.pairs, 2 * cap));
  CK(dalloc(&s.kd, cap));
  CK(dalloc(&s.vals, cap));
  CK(dalloc(&s.vals2, cap));
  CK(dalloc(&s.tmp, cap));
  CK(dalloc(&s.tmp2, cap));
  CK(dalloc(&s.chg, cap));
  CK(dalloc(&s.chg_t, cap));
  CK(dalloc(&s.flags, cap + 2));
  CK(dalloc(&s.pos, cap + 2));
  CK(dalloc(&s.seg, 2 * (cap + 2)));
  CK(dalloc(&s.tagpref, 2 * (cap + 2)));
  s.radix_hist_cap = radix_hist_words(cap) + 256;
  CK(dalloc(&s.radix_hist, s.radix_hist_cap));
  s.scan_tmp_cap = scan_tmp_words(std::max<uint64_t>(cap + 2, s.radix_hist_cap)) + 1;
  CK(dalloc(&s.scan_tmp, s.scan_tmp_cap));
  s.cap = cap;
  return PR_OK;
}

// Rebuilds adjacency A with fresh slack and at least `reserve` free tail words.
static pr_status repack_adj(Graph *g, Adj &A, uint64_t reserve) {
  const uint32_t n = g->n;
  cudaStream_t st = g->st;
  k_len_caps<<<grid_for(n), 256, 0, st>>>(A.rd, n, A.cap); count_launch();
  exclusive_scan_u32(A.cap, g->gen_tmp, n, g->scan_tmp, st);
  uint32_t last[2];
  CK(cudaMemcpyAsync(&last[0], g->gen_tmp + (n - 1), 4, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&last[1], A.cap + (n - 1), 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  uint64_t total = (uint64_t)last[0] + last[1];
  reserve = std::max<uint64_t>(reserve, std::max<uint64_t>(total / 4, 1024));
  reserve = (reserve + 3) & ~3ull;
  if (total + reserve > 0xFFFFFFFFull) {
    g->err = "graph too large: more than 2^32 - 1 column slots";
    return PR_ERR_CAPACITY;
  }
  uint32_t *nc = nullptr;
  CK(dalloc(&nc, total + reserve));
  CK(cudaMemsetAsync(nc, 0, sizeof(uint32_t) * (total + reserve), st));
  k_repack_rows<<<grid_for((uint64_t)n * 32), 256, 0, st>>>(A.rd, n, A.col, nc, g->gen_tmp); count_launch();
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  cudaFree(A.col);
  A.col = nc;
  A.col_cap = total + reserve;
  A.used = total;
  A.garbage = 0;
  return PR_OK;
}

pr_status graph_apply(Graph *g, uint64_t nd, const uint32_t *ds, const uint32_t *dd, uint64_t ni, const uint32_t *is,
                      const uint32_t *id, int nb, const uint32_t *off) {
  const uint64_t N = nd + ni;
  if (N == 0) return PR_OK;
  cudaStream_t st = g->st;
  pr_status rc = apply_scratch(g, N);
  if (rc != PR_OK) return rc;
  ApplyScratch &s = g->sc;
  const int b = g->b;
  const int kbits = 2 * b + 1;

  ApplyCtl &h = *g->actl_h;
  memset(&h, 0, sizeof(ApplyCtl));
  h.n_pend_src = g->n_pend_src;
  h.n_pend_tgt = g->n_pend_tgt;
  h.tail_out = g->out.used;
  h.tail_in = g->in.used;
  CK(cudaMemcpyAsync(g->actl, &h, sizeof(ApplyCtl), cudaMemcpyHostToDevice, st));

  k_seq_keys<<<grid_for(N), 256, 0, st>>>(ds, dd, nd, is, id, ni, nb, off, g->n, b, s.kd, s.vals, g->comp,
                                          g->inv, g->actl); count_launch();
  uint64_t *keys = s.kd;
  uint32_t *vals = s.vals;
  sort_u64_kv(&keys, &vals, s.tmp, s.vals2, N, 2 * b, s.radix_hist, s.scan_tmp, st);
  k_last_op<<<grid_for(N), 256, 0, st>>>(keys, vals, N, g->out.rd, g->out.col, b, s.flags); count_launch();
  exclusive_scan_u32(s.flags, s.pos, N, s.scan_tmp, st);
  k_emit_changes<<<grid_for(N), 256, 0, st>>>(keys, vals, N, s.flags, s.pos, b, s.chg, s.chg_t, g->actl); count_launch();
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(&h, g->actl, sizeof(ApplyCtl), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h.bad_id) {
    g->err = "vertex id out of range";
    return PR_ERR_VERTEX_RANGE;
  }
  if (h.bad_comp) {
    g->err = "a pair joins two different graphs of a batched handle";
    return PR_ERR_INVALID_ARG;
  }
  const uint32_t K = h.n_eff;
  const uint32_t K_del = h.n_eff_del;
  if (K == 0) return PR_OK;

  // the change list is already in (u, v) order (one entry per key); only the transposed
  // copy needs a sort
  uint64_t *co = s.chg;
  uint64_t *ci = sort_u64(s.chg_t, s.tmp2, K, kbits, s.radix_hist, s.scan_tmp, st);
  uint32_t *seg_o = s.seg, *seg_i = s.seg + (s.cap + 2);
  uint32_t *tp_o = s.tagpref, *tp_i = s.tagpref + (s.cap + 2);
  ApplyCtl *dctl = g->actl;
  // segments of the out-row changes
  k_seg_flags<<<grid_for(K + 1), 256, 0, st>>>(co, K, b, s.flags, tp_o); count_launch();
  exclusive_scan_u32(s.flags, s.pos, K, s.scan_tmp, st);
  exclusive_scan_u32(tp_o, tp_o, K + 1, s.scan_tmp, st);
  k_seg_emit<<<grid_for(K), 256, 0, st>>>(s.flags, s.pos, K, seg_o, &dctl->n_seg_out); count_launch();
  k_plan<<<grid_for(K), 256, 0, st>>>(g->out.rd, g->out.cap, co, K, b, seg_o, &dctl->n_seg_out, tp_o,
                                      &dctl->reloc_out, &dctl->big_cursor); count_launch();
  // segments of the in-row changes
  k_seg_flags<<<grid_for(K + 1), 256, 0, st>>>(ci, K, b, s.flags, tp_i); count_launch();
  exclusive_scan_u32(s.flags, s.pos, K, s.scan_tmp, st);
  exclusive_scan_u32(tp_i, tp_i, K + 1, s.scan_tmp, st);
  k_seg_emit<<<grid_for(K), 256, 0, st>>>(s.flags, s.pos, K, seg_i, &dctl->n_seg_in); count_launch();
  k_plan<<<grid_for(K), 256, 0, st>>>(g->in.rd, g->in.cap, ci, K, b, seg_i, &dctl->n_seg_in, tp_i,
                                      &dctl->reloc_in, &dctl->big_cursor); count_launch();
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(&h, g->actl, sizeof(ApplyCtl), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));

  // room for moved rows and staging of long rows; a repack gives rows fresh (possibly
  // smaller) slack, so the plan is redone after one
  for (int round = 0; round < 4; round++) {
    bool again = false;
    if (g->out.used + h.reloc_out > g->out.col_cap) {
      rc = repack_adj(g, g->out, 2 * h.reloc_out);
      if (rc != PR_OK) return rc;
      again = true;
    }
    if (g->in.used + h.reloc_in > g->in.col_cap) {
      rc = repack_adj(g, g->in, 2 * h.reloc_in);
      if (rc != PR_OK) return rc;
      again = true;
    }
    if (!again) break;
    CK(cudaMemsetAsync(&dctl->reloc_out, 0, 16, st));  // reloc_out, reloc_in
    CK(cudaMemsetAsync(&dctl->big_cursor, 0, 8, st));
    k_plan<<<grid_for(K), 256, 0, st>>>(g->out.rd, g->out.cap, co, K, b, seg_o, &dctl->n_seg_out, tp_o,
                                        &dctl->reloc_out, &dctl->big_cursor); count_launch();
    k_plan<<<grid_for(K), 256, 0, st>>>(g->in.rd, g->in.cap, ci, K, b, seg_i, &dctl->n_seg_in, tp_i,
                                        &dctl->reloc_in, &dctl->big_cursor); count_launch();
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&h, g->actl, sizeof(ApplyCtl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  if (h.big_cursor > g->big_cap) {
    cudaFree(g->big);
    g->big = nullptr;
    g->big_cap = 0;
    uint64_t c = std::max<uint64_t>(h.big_cursor * 2, 1u << 20);
    CK(dalloc(&g->big, c));
    g->big_cap = c;
  }
  h.tail_out = g->out.used;
  h.tail_in = g->in.used;
  h.big_cursor = 0;
  CK(cudaMemcpyAsync(&dctl->tail_out, &h.tail_out, 16, cudaMemcpyHostToDevice, st));  // tail_out, tail_in
  CK(cudaMemsetAsync(&dctl->big_cursor, 0, 8, st));

  const uint32_t lo = (uint32_t)g->p.bin_lo, hi_b = (uint32_t)g->p.bin_hi;
  const unsigned long_grid = (unsigned)std::max(1, 2 * g->sm_count);
  if (g->f32) {
    using S = Store<true>;
    RowHook<true> ho{true, g->p.alpha, (S::A *)g->adeg, (S::R *)g->R[0], (S::C *)g->C[0], (S::C *)g->C[1],
                     g->pend_src, g->pend_tgt, g->pend_cap, lo, hi_b, g->group_max, g->chunk_len, nullptr, nullptr};
    RowHook<true> hin{false,   g->p.alpha,   nullptr,      nullptr,       nullptr, nullptr, nullptr,
                      nullptr, 0,            lo,           hi_b,          g->group_max, g->chunk_len,
                      g->items, g->item_pos};
    CK(cudaMemsetAsync(&dctl->n_long, 0, 4, st));
    k_merge<true><<<K, kMergeThreads, 0, st>>>(g->out.rd, g->out.cap, g->out.col, co, b, seg_o, &dctl->n_seg_out,
                                               tp_o, &dctl->tail_out, &dctl->garbage_out, g->big, &dctl->big_cursor,
                                               g->out.col_cap, g->big_cap, dctl, ho, s.flags);
    count_launch();
    k_merge_long<true><<<long_grid, kMergeThreadsLong, 0, st>>>(g->out.rd, g->out.cap, g->out.col, co, b, seg_o,
                                               tp_o, &dctl->tail_out, &dctl->garbage_out, g->big, &dctl->big_cursor,
                                               g->out.col_cap, g->big_cap, dctl, ho, s.flags);
    count_launch();
    CK(cudaMemsetAsync(&dctl->n_long, 0, 4, st));
    k_merge<true><<<K, kMergeThreads, 0, st>>>(g->in.rd, g->in.cap, g->in.col, ci, b, seg_i, &dctl->n_seg_in, tp_i,
                                               &dctl->tail_in, &dctl->garbage_in, g->big, &dctl->big_cursor,
                                               g->in.col_cap, g->big_cap, dctl, hin, s.flags);
    count_launch();
    k_merge_long<true><<<long_grid, kMergeThreadsLong, 0, st>>>(g->in.rd, g->in.cap, g->in.col, ci, b, seg_i, tp_i,
                                               &dctl->tail_in, &dctl->garbage_in, g->big, &dctl->big_cursor,
                                               g->in.col_cap, g->big_cap, dctl, hin, s.flags);
    count_launch();
  } else {
    using S = Store<false>;
    RowHook<false> ho{true, g->p.alpha, (S::A *)g->adeg, (S::R *)g->R[0], (S::C *)g->C[0], (S::C *)g->C[1],
                      g->pend_src, g->pend_tgt, g->pend_cap, lo, hi_b, g->group_max, g->chunk_len, nullptr, nullptr};
    RowHook<false> hin{false,   g->p.alpha,   nullptr,      nullptr,       nullptr, nullptr, nullptr,
                       nullptr, 0,            lo,           hi_b,          g->group_max, g->chunk_len,
                       g->items, g->item_pos};
    CK(cudaMemsetAsync(&dctl->n_long, 0, 4, st));
    k_merge<false><<<K, kMergeThreads, 0, st>>>(g->out.rd, g->out.cap, g->out.col, co, b, seg_o, &dctl->n_seg_out,
                                                tp_o, &dctl->tail_out, &dctl->garbage_out, g->big, &dctl->big_cursor,
                                                g->out.col_cap, g->big_cap, dctl, ho, s.flags);
    count_launch();
    k_merge_long<false><<<long_grid, kMergeThreadsLong, 0, st>>>(g->out.rd, g->out.cap, g->out.col, co, b, seg_o,
                                                tp_o, &dctl->tail_out, &dctl->garbage_out, g->big, &dctl->big_cursor,
                                                g->out.col_cap, g->big_cap, dctl, ho, s.flags);
    count_launch();
    CK(cudaMemsetAsync(&dctl->n_long, 0, 4, st));
    k_merge<false><<<K, kMergeThreads, 0, st>>>(g->in.rd, g->in.cap, g->in.col, ci, b, seg_i, &dctl->n_seg_in, tp_i,
                                                &dctl->tail_in, &dctl->garbage_in, g->big, &dctl->big_cursor,
                                                g->in.col_cap, g->big_cap, dctl, hin, s.flags);
    count_launch();
    k_merge_long<false><<<long_grid, kMergeThreadsLong, 0, st>>>(g->in.rd, g->in.cap, g->in.col, ci, b, seg_i, tp_i,
                                                &dctl->tail_in, &dctl->garbage_in, g->big, &dctl->big_cursor,
                                                g->in.col_cap, g->big_cap, dctl, hin, s.flags);
    count_launch();
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(&h, g->actl, sizeof(ApplyCtl), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h.overflow) {
    g->err = "internal error: no room for a moved row (graph rows partly updated)";
    return PR_ERR_CUDA;
  }

  g->m = g->m + (uint64_t)(K - K_del) - (uint64_t)K_del;
  g->out.used = h.tail_out;
  g->in.used = h.tail_in;
  g->out.garbage += h.garbage_out;
  g->in.garbage += h.garbage_in;
  g->n_pend_src = std::min(h.n_pend_src, g->pend_cap);
  g->n_pend_tgt = std::min(h.n_pend_tgt, g->pend_cap);
  if (h.n_pend_src > g->pend_cap || h.n_pend_tgt > g->pend_cap) g->pend_all = true;
  if (h.dead_changed) g->dead_dirty = true;
  if (h.bins_changed) g->ident_dirty = true;
  // give abandoned slots back once they dominate
  if (g->out.garbage > g->out.used / 2 && g->out.garbage > 1024) {
    rc = repack_adj(g, g->out, 0);
    if (rc != PR_OK) return rc;
  }
  if (g->in.garbage > g->in.used / 2 && g->in.garbage > 1024) {
    rc = repack_adj(g, g->in, 0);
    if (rc != PR_OK) return rc;
  }
  // the degree-binned vertex order used by full and dense sweeps follows the graph
  return graph_refresh_ident(g);
}

pr_status graph_export(Graph *g, int dir, uint64_t *offs_h, uint32_t *cols_h) {
  const uint32_t n = g->n;
  cudaStream_t st = g->st;
  Adj &A = dir ? g->in : g->out;
  k_row_len<<<grid_for((uint64_t)n + 1), 256, 0, st>>>(A.rd, n, g->gen_tmp); count_launch();
  exclusive_scan_u32(g->gen_tmp, g->gen_tmp2, (uint64_t)n + 1, g->scan_tmp, st);
  uint32_t *packed = nullptr;
  CK(dalloc(&packed, std::max<uint64_t>(g->m, 1)));
  k_pack_rows<<<grid_for((uint64_t)n * 32), 256, 0, st>>>(A.rd, n, A.col, g->gen_tmp2, packed); count_launch();
  std::vector<uint32_t> off(n + 1);
  std::vector<uint32_t> icols;
  if (g->perm) icols.resize(g->m);
  uint32_t *dst_cols = g->perm ? icols.data() : cols_h;
  cudaError_t e = cudaMemcpyAsync(off.data(), g->gen_tmp2, 4ull * (n + 1), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dst_cols, packed, 4ull * g->m, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(packed);
  if (e != cudaSuccess) return cuda_fail(g, e, "export csr");
  if (!g->perm) {
    for (uint32_t v = 0; v <= n; v++) offs_h[v] = off[v];
    return PR_OK;
  }
  // rows and columns back in the caller's numbering, each row sorted
  const std::vector<uint32_t> &perm = g->perm_h;
  std::vector<uint32_t> inv(n);
  for (uint32_t r = 0; r < n; r++) inv[perm[r]] = r;
  uint64_t at = 0;
  for (uint32_t v = 0; v < n; v++) {
    offs_h[v] = at;
    const uint32_t r = inv[v];
    for (uint32_t j = off[r]; j < off[r + 1]; j++) cols_h[at++] = perm[icols[j]];
    std::sort(cols_h + offs_h[v], cols_h + at);
  }
  offs_h[n] = at;
  return PR_OK;
}

pr_status graph_refresh_ident(Graph *g) {
  if (!g->ident_dirty) return PR_OK;
  const uint32_t n = g->n;
  cudaStream_t st = g->st;
  uint32_t *over = (uint32_t *)&g->actl->n_seg_out;  // reuse a device word
  const uint32_t lo = (uint32_t)g->p.bin_lo, gmax = g->group_max, chunk = g->chunk_len;
  const uint32_t nblk = (uint32_t)(((uint64_t)n + kIdentTile - 1) / kIdentTile);
  const uint64_t len = 4ull * nblk + 2;  // tiers 0-2, 0, chunk counts, 0 (<= n + 8: fits gen_tmp)
  CK(cudaMemsetAsync(over, 0, 4, st));
  k_tier_counts<<<nblk, 256, 0, st>>>(g->in.rd, n, lo, gmax, chunk, nblk, g->gen_tmp, over);
  count_launch();
  exclusive_scan_u32(g->gen_tmp, g->gen_tmp2, len, g->scan_tmp, st);
  uint32_t h[4] = {0, 0, 0, 0};  // tier-0 count, tiers 0+1, n + chunk items, over
  CK(cudaMemcpyAsync(&h[0], g->gen_tmp2 + nblk, 4, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&h[1], g->gen_tmp2 + 2 * nblk, 4, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&h[2], g->gen_tmp2 + len - 1, 4, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&h[3], over, 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h[3]) {
    g->err = "a vertex has more in-edges than 2^21 sweep chunks hold (raise chunk_len)";
    return PR_ERR_CAPACITY;
  }
  const uint32_t c01 = h[1], total = h[2] - n;
  if ((uint64_t)c01 + total > g->items_cap || total > g->chunk_cap) {  // items, and partials by chunk number
    cudaFree(g->items);
    cudaFree(g->items_cmp);
    cudaFree(g->partials);
    g->items = g->items_cmp = nullptr;
    g->partials = nullptr;
    g->items_cap = g->chunk_cap = 0;
    uint64_t chunks = (uint64_t)total + total / 4 + 1024;
    uint64_t cap = (uint64_t)n + chunks;
    CK(dalloc(&g->items, cap));
    CK(dalloc(&g->items_cmp, cap));
    CK(cudaMalloc(&g->partials, 8 * chunks));
    g->items_cap = cap;
    g->chunk_cap = chunks;
  }
  k_items_write<<<nblk, 256, 0, st>>>(g->in.rd, n, lo, gmax, chunk, nblk, g->gen_tmp2, g->items, g->item_pos);
  count_launch();
  CK(cudaGetLastError());
  g->item_cnt[0] = h[0];
  g->item_cnt[1] = c01 - h[0];
  g->item_cnt[2] = total;
  g->ident_dirty = false;
  return PR_OK;
}

pr_status graph_refresh_dead(Graph *g) {
  if (!g->dead_dirty) return PR_OK;
  const uint32_t n = g->n;
  cudaStream_t st = g->st;
  uint32_t *cnt = (uint32_t *)&g->actl->n_seg_in;
  k_dead_flags<<<grid_for(n), 256, 0, st>>>(g->out.rd, n, g->gen_tmp); count_launch();
  exclusive_scan_u32(g->gen_tmp, g->gen_tmp2, n, g->scan_tmp, st);
  k_compact_ids<<<grid_for(n), 256, 0, st>>>(g->gen_tmp, g->gen_tmp2, n, g->dead, cnt); count_launch();
  uint32_t c = 0;
  CK(cudaMemcpyAsync(&c, cnt, 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  g->n_dead = c;
  g->dead_dirty = false;
  return PR_OK;
}

__global__ void k_fill_comp(uint16_t *comp, uint32_t first, uint32_t count, uint16_t c) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) comp[first + i] = c;
}

// One thread per vertex: flags an out-edge that leaves the vertex's graph.
__global__ void k_check_comp(const uint2 *rd, const uint32_t *col, const uint16_t *comp, uint32_t n, uint32_t *bad) {
  uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  uint2 d = rd[u];
  for (uint32_t j = 0; j < d.y; j++)
    if (comp[col[d.x + j]] != comp[u]) {
      atomicOr(bad, 1u);
      return;
    }
}

template <bool F32>
__global__ void k_init_comp_rank(const uint16_t *comp, uint32_t n, const typename Store<F32>::R *init,
                                 const typename Store<F32>::A *adeg, typename Store<F32>::R *R0,
                                 typename Store<F32>::R *R1, typename Store<F32>::C *C0, typename Store<F32>::C *C1) {
  using S = Store<F32>;
  uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  typename S::R r = init[comp[v]];
  typename S::C c = S::contrib(r, adeg[v]);
  R0[v] = r;
  R1[v] = r;
  C0[v] = c;
  C1[v] = c;
}

template <bool F32>
__global__ void k_comp_consts(const uint32_t *first, uint32_t ncomp, double alpha, typename Store<F32>::R *base,
                              typename Store<F32>::R *init) {
  using S = Store<F32>;
  uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncomp) return;
  double nc = (double)(first[c + 1] - first[c]);
  base[c] = S::from_double((1.0 - alpha) / nc);
  init[c] = S::from_double(1.0 / nc);
}

pr_status components_setup(Graph *g, const std::vector<uint32_t> &comp_n) {
  const uint32_t n = g->n, nc = (uint32_t)comp_n.size();
  cudaStream_t st = g->st;
  g->ncomp = nc;
  g->comp_first.assign(nc + 1, 0);
  for (uint32_t c = 0; c < nc; c++) g->comp_first[c + 1] = g->comp_first[c] + comp_n[c];
  CK(dalloc(&g->comp, n));
  for (uint32_t c = 0; c < nc; c++) {
    k_fill_comp<<<grid_for(comp_n[c]), 256, 0, st>>>(g->comp, g->comp_first[c], comp_n[c], (uint16_t)c);
    count_launch();
  }
  uint32_t *bad = nullptr, *first_d = nullptr;
  CK(dalloc(&bad, 1));
  CK(dalloc(&first_d, nc + 1));
  CK(cudaMemsetAsync(bad, 0, 4, st));
  CK(cudaMemcpyAsync(first_d, g->comp_first.data(), 4ull * (nc + 1), cudaMemcpyHostToDevice, st));
  k_check_comp<<<grid_for(n), 256, 0, st>>>(g->out.rd, g->out.col, g->comp, n, bad);
  count_launch();
  uint32_t hbad = 0;
  CK(cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  cudaFree(bad);
  if (hbad) {
    cudaFree(first_d);
    g->err = "an edge joins two different graphs of a batched handle";
    return PR_ERR_INVALID_ARG;
  }
  CK(cudaMalloc(&g->comp_base, 8ull * nc));
  CK(cudaMalloc(&g->comp_init, 8ull * nc));
  CK(dalloc(&g->dRc, 3ull * nc));
  CK(dalloc(&g->comp_out, 4ull * nc));
  CK(dalloc(&g->comp_last, nc));
  if (g->f32) {
    using S = Store<true>;
    k_comp_consts<true><<<grid_for(nc), 256, 0, st>>>(first_d, nc, g->p.alpha, (S::R *)g->comp_base, (S::R *)g->comp_init);
    count_launch();
    k_init_comp_rank<true><<<grid_for(n), 256, 0, st>>>(g->comp, n, (const S::R *)g->comp_init, (const S::A *)g->adeg,
                                                        (S::R *)g->R[0], (S::R *)g->R[1], (S::C *)g->C[0],
                                                        (S::C *)g->C[1]);
  } else {
    using S = Store<false>;
    k_comp_consts<false><<<grid_for(nc), 256, 0, st>>>(first_d, nc, g->p.alpha, (S::R *)g->comp_base,
                                                       (S::R *)g->comp_init);
    count_launch();
    k_init_comp_rank<false><<<grid_for(n), 256, 0, st>>>(g->comp, n, (const S::R *)g->comp_init,
                                                         (const S::A *)g->adeg, (S::R *)g->R[0], (S::R *)g->R[1],
                                                         (S::C *)g->C[0], (S::C *)g->C[1]);
  }
  count_launch();
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  cudaFree(first_d);
  g->comp_stats.assign(nc, pr_stats{});
  return PR_OK;
}

void graph_free(Graph *g) {
  Adj *adjs[2] = {&g->out, &g->in};
  for (Adj *A : adjs) {
    cudaFree(A->rd);
    cudaFree(A->cap);
    cudaFree(A->col);
  }
  for (int i = 0; i < 2; i++) {
    cudaFree(g->R[i]);
    cudaFree(g->C[i]);
  }
  cudaFree(g->adeg);
  cudaFree(g->bitmap);
  cudaFree(g->xbits);
  cudaFree(g->stamp);
  cudaFree(g->items);
  cudaFree(g->items_cmp);
  cudaFree(g->item_pos);
  cudaFree(g->hub_v);
  cudaFree(g->hub_base);
  cudaFree(g->comp);
  cudaFree(g->comp_base);
  cudaFree(g->comp_init);
  cudaFree(g->dRc);
  cudaFree(g->comp_out);
  cudaFree(g->comp_last);
  cudaFree(g->partials);
  cudaFree(g->chunk_done);
  for (int i = 0; i < 3; i++) cudaFree(g->list[i]);
  cudaFree(g->xlist);
  cudaFree(g->dead);
  cudaFree(g->pend_src);
  cudaFree(g->pend_tgt);
  cudaFree(g->ctl);
  if (g->ctl_h) cudaFreeHost(g->ctl_h);
  cudaFree(g->dpart);
  ApplyScratch &s = g->sc;
  cudaFree(s.pairs); cudaFree(s.kd); cudaFree(s.vals); cudaFree(s.vals2); cudaFree(s.tmp); cudaFree(s.tmp2);
  cudaFree(s.boff);
  cudaFree(s.chg); cudaFree(s.chg_t); cudaFree(s.flags); cudaFree(s.pos); cudaFree(s.seg);
  cudaFree(s.tagpref); cudaFree(s.radix_hist); cudaFree(s.scan_tmp);
  cudaFree(g->actl);
  if (g->actl_h) cudaFreeHost(g->actl_h);
  cudaFree(g->big);
  cudaFree(g->gen_tmp);
  cudaFree(g->gen_tmp2);
  cudaFree(g->perm);
  cudaFree(g->inv);
  cudaFree(g->scan_tmp);
  if (g->cg_exec) cudaGraphExecDestroy(g->cg_exec);
  if (g->cg) cudaGraphDestroy(g->cg);
  if (g->ev0) cudaEventDestroy(g->ev0);
  if (g->ev1) cudaEventDestroy(g->ev1);
}

}  // namespace prdf

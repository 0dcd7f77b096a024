// order.cu - the internal vertex numbering of single-graph handles.
//
// The sweeps gather one contribution per in-edge, and their cost is the number of distinct
// 32-byte sectors those gathers touch.  A breadth-first numbering (over out- and in-edges
// together) gives the vertices discovered from one vertex consecutive numbers, so the
// short rows that a warp sweeps side by side gather from nearby contributions.  Two are
// computed, from different first levels:
//  kOrderFromMax: the vertex of largest degree (graphs with hubs, such as R-MAT: its
//    neighbourhood is most of the graph within a few levels);
//  kOrderFromSeeds: max(kSeeds, n / kSeedCell) vertices evenly spaced in the caller's
//    numbering (graphs of large diameter, such as chains of k-mers, which one seed would
//    cover only at one level per few dozen vertices).
//  kOrderPerGraph (batched handles): the vertex of largest degree of every graph, then a
//    stable sort by graph, so that each graph keeps its id range and within it the order
//    of its own breadth-first search from that vertex.
// Level by level, a newly reached vertex takes its place after the vertices reached from
// earlier-numbered vertices of the previous level (the earliest adjacent one decides),
// ties by vertex id; vertices not reached within kMaxLevels levels follow in id order.
// Each level costs a few launches and one host synchronisation.  A handle keeps the
// numbering whose modelled short-row gathers (order_cost) touch the fewest sectors, if
// that is at least 5% fewer than under the caller's numbering: a grid numbered row by row
// already gathers consecutive contributions.  (Putting the vertices of largest out-degree
// side by side was measured slower: a fifth of the gathers then fall in one 64 KB run,
// whose few L2 slices serve them while the others wait.)  Ranks, results and the update
// semantics do not depend on the numbering: ids are translated at the boundary (batches,
// ranks in and out, affected sets, CSR export).
#include <algorithm>
#include <cstdint>

#include "prdf_graph.cuh"

namespace prdf {

#define CK(call)                                            \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(g, e_, #call);  \
  } while (0)

namespace {

constexpr uint32_t kUnset = 0xFFFFFFFFu;
constexpr int kMaxLevels = 1024;
constexpr uint32_t kSeeds = 8192;     // at least this many seeds,
constexpr uint32_t kSeedCell = 2048;  // and one per this many vertices (a cell of a few hundred levels at most)

__global__ void k_order_init(uint32_t n, uint32_t *label, uint32_t *cand) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) {
    label[v] = kUnset;
    cand[v] = kUnset;
  }
}

// the vertex of largest out + in degree (smallest id on ties): a max of (degree << 32 | ~v)
__global__ void k_order_seed(const uint2 *out_rd, const uint2 *in_rd, uint32_t n, unsigned long long *best) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long key = 0;
  if (v < n) key = ((unsigned long long)(out_rd[v].y + in_rd[v].y) << 32) | (unsigned long long)(~v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, key, o);
    key = y > key ? y : key;
  }
  if ((threadIdx.x & 31) == 0 && key) atomicMax(best, key);
}

__global__ void k_order_start(const unsigned long long *best, uint32_t *label, uint32_t *perm) {
  const uint32_t s = ~(uint32_t)(*best & 0xFFFFFFFFull);
  label[s] = 0;
  perm[0] = s;
}

// graph of each vertex (first[c] <= v < first[c + 1]; nc <= kMaxComponents)
__global__ void k_order_graph_of(const uint32_t *first, uint32_t nc, uint32_t n, uint32_t *gid) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  uint32_t lo = 0, hi = nc;  // last c with first[c] <= v
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (first[mid] <= v) lo = mid; else hi = mid;
  }
  gid[v] = lo;
}

// every graph's vertex of largest out + in degree (smallest id on ties)
__global__ void k_order_graph_seed(const uint2 *out_rd, const uint2 *in_rd, const uint32_t *gid, uint32_t n,
                                   unsigned long long *best) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) atomicMax(best + gid[v], ((unsigned long long)(out_rd[v].y + in_rd[v].y) << 32) | (unsigned long long)(~v));
}

// level 0 of kOrderPerGraph: the graphs' seeds in graph order (graphs without vertices
// have none); one thread
__global__ void k_order_graph_start(const unsigned long long *best, uint32_t nc, uint32_t *label, uint32_t *perm,
                                    uint32_t *count) {
  uint32_t k = 0;
  for (uint32_t c = 0; c < nc; c++) {
    if (!best[c]) continue;
    const uint32_t s = ~(uint32_t)(best[c] & 0xFFFFFFFFull);
    label[s] = k;
    perm[k++] = s;
  }
  *count = k;
}

// sort keys of the final order: graph, then breadth-first number
__global__ void k_order_graph_keys(const uint32_t *gid, const uint32_t *label, uint32_t n, unsigned long long *keys) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) keys[v] = ((unsigned long long)gid[v] << 32) | label[v];
}

__global__ void k_order_graph_perm(const unsigned long long *sorted, const uint32_t *rank_perm, uint32_t n,
                                   uint32_t *perm, uint32_t *inv) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const uint32_t v = rank_perm[(uint32_t)(sorted[i] & 0xFFFFFFFFull)];
    perm[i] = v;
    inv[v] = i;
  }
}

// level 0 of kOrderFromSeeds: seed i is vertex i * step
__global__ void k_order_seeds(uint32_t k, uint32_t step, uint32_t *label, uint32_t *perm) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) {
    label[i * step] = i;
    perm[i] = i * step;
  }
}

// One level: every vertex of the frontier (perm[lo, hi), numbered lo..hi-1) offers its
// number to its unnumbered neighbours (out- and in-rows, one warp per frontier vertex); a
// neighbour keeps the smallest offer, and its first offer lists it.
__global__ void k_order_expand(const uint2 *out_rd, const uint32_t *out_col, const uint2 *in_rd,
                               const uint32_t *in_col, const uint32_t *perm, uint32_t lo, uint32_t hi,
                               const uint32_t *label, uint32_t *cand, uint32_t *next, uint32_t *cnt) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t k = lo + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5); k < hi; k += nwarps) {
    const uint32_t u = perm[k];
    for (int dir = 0; dir < 2; dir++) {
      const uint2 d = dir ? in_rd[u] : out_rd[u];
      const uint32_t *col = (dir ? in_col : out_col) + d.x;
      for (uint32_t j = lane; j < d.y; j += 32) {
        const uint32_t w = col[j];
        if (label[w] != kUnset) continue;
        const uint32_t old = atomicMin(&cand[w], k);
        if (old == kUnset) next[atomicAdd(cnt, 1u)] = w;
      }
    }
  }
}

__global__ void k_order_keys(const uint32_t *next, uint32_t cnt, const uint32_t *cand, unsigned long long *keys) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) keys[i] = ((unsigned long long)cand[next[i]] << 32) | next[i];
}

__global__ void k_order_assign(const unsigned long long *keys, uint32_t cnt, uint32_t base, uint32_t *label,
                               uint32_t *perm) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) {
    const uint32_t w = (uint32_t)(keys[i] & 0xFFFFFFFFull);
    label[w] = base + i;
    perm[base + i] = w;
  }
}

__global__ void k_order_unset_flags(const uint32_t *label, uint32_t n, uint32_t *flags) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) flags[v] = label[v] == kUnset ? 1u : 0u;
}

__global__ void k_order_rest(const uint32_t *flags, const uint32_t *pos, uint32_t n, uint32_t base, uint32_t *label,
                             uint32_t *perm) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n && flags[v]) {
    label[v] = base + pos[v];
    perm[base + pos[v]] = v;
  }
}

// The gather cost model that decides whether the new numbering is kept: the rows of at
// most kScoreRowMax in-edges are swept 32 consecutive rows a warp, one in-edge per lane per
// step, as the short-row tiers do; each step costs one request per distinct 32-byte sector
// among the lanes' contributions.  cnt[0] sums those sectors under the caller's
// numbering, cnt[1] under the new one.  (Long rows gather about one sector per in-edge in
// any numbering: their in-neighbours are spread over the graph.)
constexpr uint32_t kScoreRowMax = 64;

__global__ void k_order_score(const uint2 *in_rd, const uint32_t *in_col, const uint32_t *perm,
                              const uint32_t *inv, uint32_t n, int sec_shift, unsigned long long *cnt) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t ngroups = (uint32_t)(((uint64_t)n + 31) / 32);
  unsigned long long sec[2] = {0, 0};
  for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < ngroups; w += nwarps) {
    const uint32_t pos = w * 32 + lane;
    for (int mode = 0; mode < 2; mode++) {
      uint2 d = make_uint2(0, 0);
      if (pos < n) {
        d = in_rd[mode ? perm[pos] : pos];
        if (d.y > kScoreRowMax) d.y = 0;
      }
      uint32_t dmax = d.y;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      for (uint32_t k = 0; k < dmax; k++) {
        const bool act = k < d.y;
        const unsigned am = __ballot_sync(0xffffffffu, act);
        if (act) {
          uint32_t c = in_col[d.x + k];
          if (mode) c = inv[c];
          const unsigned peers = __match_any_sync(am, c >> sec_shift);
          if ((uint32_t)(__ffs(peers) - 1) == lane) sec[mode]++;
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sec[0] += __shfl_xor_sync(0xffffffffu, sec[0], o);
    sec[1] += __shfl_xor_sync(0xffffffffu, sec[1], o);
  }
  if (lane == 0) {
    if (sec[0]) atomicAdd(&cnt[0], sec[0]);
    if (sec[1]) atomicAdd(&cnt[1], sec[1]);
  }
}

__global__ void k_map_ids(const uint32_t *inv, uint32_t *a, uint64_t m) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) a[i] = inv[a[i]];
}

unsigned grid_of(uint64_t n) { return (unsigned)std::max<uint64_t>(1, (n + 255) / 256); }

}  // namespace

pr_status vertex_order(Graph *g, int kind, uint32_t *perm, uint32_t *inv, const std::vector<uint32_t> *comp_n) {
  const uint32_t n = g->n;
  cudaStream_t st = g->st;
  pr_status rc = apply_scratch(g, n);
  if (rc != PR_OK) return rc;
  ApplyScratch &s = g->sc;
  uint32_t *cand = s.flags, *next = s.pos, *cnt = (uint32_t *)&g->actl->n_seg_out;
  unsigned long long *keys = (unsigned long long *)s.kd;
  k_order_init<<<grid_of(n), 256, 0, st>>>(n, inv, cand);
  count_launch();
  int b = 0;
  while (b < 32 && (1ull << b) < (uint64_t)n) b++;
  uint32_t lo = 0, hi;
  uint32_t *gid = nullptr;
  if (kind == kOrderPerGraph) {
    // graphs of a batched handle: one seed each
    const uint32_t nc = comp_n ? (uint32_t)comp_n->size() : 0u;
    if (!nc || nc > kMaxComponents) {
      g->err = "per-graph numbering needs the graphs' sizes";
      return PR_ERR_INVALID_ARG;
    }
    std::vector<uint32_t> first(nc + 1, 0);
    for (uint32_t c = 0; c < nc; c++) first[c + 1] = first[c] + (*comp_n)[c];
    uint32_t *first_d = g->gen_tmp;  // needed only until every vertex has its graph
    unsigned long long *best = (unsigned long long *)s.tmp2;
    CK(cudaMemcpyAsync(first_d, first.data(), 4ull * (nc + 1), cudaMemcpyHostToDevice, st));
    k_order_graph_of<<<grid_of(n), 256, 0, st>>>(first_d, nc, n, s.vals);
    count_launch();
    gid = s.vals;
    CK(cudaMemsetAsync(best, 0, 8ull * nc, st));
    k_order_graph_seed<<<grid_of(n), 256, 0, st>>>(g->out.rd, g->in.rd, gid, n, best);
    count_launch();
    k_order_graph_start<<<1, 1, 0, st>>>(best, nc, inv, perm, cnt);
    count_launch();
    CK(cudaMemcpyAsync(&hi, cnt, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  } else if (kind == kOrderFromSeeds) {
    const uint32_t k = std::min(n, std::max(kSeeds, n / kSeedCell)), step = n / k;
    k_order_seeds<<<grid_of(k), 256, 0, st>>>(k, step, inv, perm);
    count_launch();
    hi = k;
  } else {
    unsigned long long *best = (unsigned long long *)s.tmp2;
    CK(cudaMemsetAsync(best, 0, 8, st));
    k_order_seed<<<grid_of(n), 256, 0, st>>>(g->out.rd, g->in.rd, n, best);
    count_launch();
    k_order_start<<<1, 1, 0, st>>>(best, inv, perm);
    count_launch();
    hi = 1;
  }
  const unsigned egrid = (unsigned)std::max(1, g->sm_count * 8);
  for (int level = 0; hi > lo && level < kMaxLevels; level++) {
    CK(cudaMemsetAsync(cnt, 0, 4, st));
    k_order_expand<<<egrid, 256, 0, st>>>(g->out.rd, g->out.col, g->in.rd, g->in.col, perm, lo, hi, inv, cand,
                                          next, cnt);
    count_launch();
    uint32_t c = 0;
    CK(cudaMemcpyAsync(&c, cnt, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (c) {
      k_order_keys<<<grid_of(c), 256, 0, st>>>(next, c, cand, keys);
      count_launch();
      // keys: (offering number < n: b bits) << 32 | vertex id
      uint64_t *sorted = sort_u64((uint64_t *)keys, s.tmp, c, 32 + b, s.radix_hist, s.scan_tmp, st);
      k_order_assign<<<grid_of(c), 256, 0, st>>>((const unsigned long long *)sorted, c, hi, inv, perm);
      count_launch();
    }
    lo = hi;
    hi += c;
  }
  if (hi < n) {
    // vertices no edge path reaches from the first level, or none within kMaxLevels, in id order
    k_order_unset_flags<<<grid_of(n), 256, 0, st>>>(inv, n, g->gen_tmp);
    count_launch();
    exclusive_scan_u32(g->gen_tmp, g->gen_tmp2, n, g->scan_tmp, st);
    k_order_rest<<<grid_of(n), 256, 0, st>>>(g->gen_tmp, g->gen_tmp2, n, hi, inv, perm);
    count_launch();
  }
  if (kind == kOrderPerGraph) {
    // stable by graph: each graph keeps its id range, ordered by its own search
    const uint32_t nc = (uint32_t)comp_n->size();
    int cb = 1;
    while ((1u << cb) < nc) cb++;
    k_order_graph_keys<<<grid_of(n), 256, 0, st>>>(gid, inv, n, keys);
    count_launch();
    const unsigned long long *sorted =
        (const unsigned long long *)sort_u64((uint64_t *)keys, s.tmp, n, 32 + cb, s.radix_hist, s.scan_tmp, st);
    CK(cudaMemcpyAsync(next, perm, 4ull * n, cudaMemcpyDeviceToDevice, st));
    k_order_graph_perm<<<grid_of(n), 256, 0, st>>>(sorted, next, n, perm, inv);
    count_launch();
  }

  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return PR_OK;
}

pr_status order_cost(Graph *g, const uint32_t *perm, const uint32_t *inv, uint64_t cost[2]) {
  cudaStream_t st = g->st;
  const uint32_t n = g->n;
  unsigned long long *cnt = (unsigned long long *)g->sc.tmp2, h[2] = {0, 0};
  CK(cudaMemsetAsync(cnt, 0, 16, st));
  const unsigned grid = (unsigned)std::max(1, g->sm_count * 8);
  // 8-byte contributions: 4 to a sector; 4-byte: 8
  k_order_score<<<grid, 256, 0, st>>>(g->in.rd, g->in.col, perm, inv, n, g->f32 ? 3 : 2, cnt);
  count_launch();
  CK(cudaMemcpyAsync(h, cnt, 16, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  cost[0] = h[0];
  cost[1] = h[1];
  return PR_OK;
}

void map_ids(const uint32_t *inv, uint32_t *a, uint64_t m, cudaStream_t st) {
  if (m == 0) return;
  k_map_ids<<<grid_of(m), 256, 0, st>>>(inv, a, m);
  count_launch();
}

}  // namespace prdf

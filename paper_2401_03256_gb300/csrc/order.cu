// order.cu - the internal vertex numbering of single-graph handles.
//
// The sweeps gather one contribution per in-edge, and their cost is the number of distinct
// 32-byte sectors those gathers touch.  A breadth-first numbering from the vertex of
// largest degree (over out- and in-edges together) gives the vertices discovered from one
// vertex consecutive numbers, so the short rows that a warp sweeps side by side gather
// from nearby contributions; on R-MAT scale 22 a full sweep takes 8% less time than under a
// random numbering.  The numbering is deterministic: level by level, a newly reached vertex
// takes its place after the vertices reached from earlier-numbered vertices of the
// previous level (the earliest adjacent one decides), ties by vertex id; vertices not
// reached within kMaxLevels levels follow in id order.  Each level costs a few launches and
// one host synchronisation, so graphs of huge diameter (chains of k-mers: one level per
// few dozen vertices) keep their own numbering past the cap instead of paying seconds at
// creation.  Ranks, results and the update semantics do not depend on the numbering: ids
// are translated at the boundary (batches, ranks in and out, affected sets, CSR export).
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

__global__ void k_map_ids(const uint32_t *inv, uint32_t *a, uint64_t m) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) a[i] = inv[a[i]];
}

unsigned grid_of(uint64_t n) { return (unsigned)std::max<uint64_t>(1, (n + 255) / 256); }

}  // namespace

pr_status vertex_order(Graph *g, uint32_t *perm, uint32_t *inv) {
  const uint32_t n = g->n;
  cudaStream_t st = g->st;
  pr_status rc = apply_scratch(g, n);
  if (rc != PR_OK) return rc;
  ApplyScratch &s = g->sc;
  uint32_t *cand = s.flags, *next = s.pos, *cnt = (uint32_t *)&g->actl->n_seg_out;
  unsigned long long *keys = (unsigned long long *)s.kd, *best = (unsigned long long *)s.tmp2;
  k_order_init<<<grid_of(n), 256, 0, st>>>(n, inv, cand);
  count_launch();
  CK(cudaMemsetAsync(best, 0, 8, st));
  k_order_seed<<<grid_of(n), 256, 0, st>>>(g->out.rd, g->in.rd, n, best);
  count_launch();
  k_order_start<<<1, 1, 0, st>>>(best, inv, perm);
  count_launch();
  int b = 0;
  while (b < 32 && (1ull << b) < (uint64_t)n) b++;
  uint32_t lo = 0, hi = 1;
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
    // vertices no edge path reaches from the seed, or none within kMaxLevels, in id order
    k_order_unset_flags<<<grid_of(n), 256, 0, st>>>(inv, n, g->gen_tmp);
    count_launch();
    exclusive_scan_u32(g->gen_tmp, g->gen_tmp2, n, g->scan_tmp, st);
    k_order_rest<<<grid_of(n), 256, 0, st>>>(g->gen_tmp, g->gen_tmp2, n, hi, inv, perm);
    count_launch();
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return PR_OK;
}

void map_ids(const uint32_t *inv, uint32_t *a, uint64_t m, cudaStream_t st) {
  if (m == 0) return;
  k_map_ids<<<grid_of(m), 256, 0, st>>>(inv, a, m);
  count_launch();
}

}  // namespace prdf

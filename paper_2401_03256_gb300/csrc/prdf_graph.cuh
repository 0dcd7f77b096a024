// prdf_graph.cuh - the graph handle behind the opaque pr_graph of the C ABI.
#pragma once

#include <string>
#include <vector>

#include "prdf_common.cuh"
#include "../../include/prdf.h"

namespace prdf {

// Rows get room to grow: cap = round4(len + 2 + len / 8) at build / repack time,
// round4(2 len + 2) when a row outgrows its slots and moves to the free tail.
__host__ __device__ inline uint32_t slack_cap(uint32_t len) {
  uint64_t c = (uint64_t)len + 2 + len / 8;
  return (uint32_t)((c + 3) & ~3ull);
}
__host__ __device__ inline uint32_t move_cap(uint32_t len) {
  uint64_t c = 2ull * len + 2;
  return (uint32_t)((c + 3) & ~3ull);
}

struct Graph {
  int device = 0;
  cudaStream_t st = nullptr;
  int sm_count = 0;
  uint32_t n = 0;
  int b = 1;             // bits of a vertex id in packed keys
  uint64_t m = 0;        // stored edges (self-loops included)
  pr_params p{};
  bool f32 = false;
  bool teleport = false;

  Adj out, in;
  void *R[2] = {nullptr, nullptr};   // ranks, both parities equal between calls
  void *C[2] = {nullptr, nullptr};   // contributions alpha R[u] / |out(u)|
  void *adeg = nullptr;              // alpha / |out(u)| (0 for a dead end)
  uint32_t *bitmap = nullptr;        // affected flags, all zero between calls
  uint32_t *xbits = nullptr;         // out-row scanned in this call, all zero between calls
  uint16_t *stamp = nullptr;         // iteration a vertex joins the affected set, 0xFFFF between calls
  uint32_t *list[3] = {nullptr, nullptr, nullptr};  // affected vertices by in-degree bin
  uint32_t *xlist = nullptr;         // vertices a continuation launch recorded for expansion
  bool ident_dirty = true;
  // internal numbering (single-graph handles): perm[internal] = caller's id, inv the inverse;
  // null when the handle keeps the caller's numbering
  uint32_t *perm = nullptr, *inv = nullptr;
  std::vector<uint32_t> perm_h;
  // Sweep items (16 B each) in tier order: tier 0 and 1 items {v, start, len, 0}, then the
  // chunk_len-edge chunks of tier-2 rows {v, start of chunk, len | index in row << 10 |
  // several-chunks flag << 31, chunk number}.  items_cmp holds the affected subset during
  // dense Dynamic Frontier iterations.
  uint4 *items = nullptr, *items_cmp = nullptr;
  uint64_t items_cap = 0;
  uint32_t item_cnt[3] = {0, 0, 0};  // tier-0 items, tier-1 items, chunks
  uint32_t *item_pos = nullptr;      // per vertex: index of its (first) item
  uint64_t chunk_cap = 0;
  void *partials = nullptr;          // one contribution-typed partial sum per chunk
  uint32_t *chunk_done = nullptr;    // per vertex: chunks finished in this iteration (0 between)
  uint32_t *hub_v = nullptr;         // long out-rows queued for cooperative marking (per slot)
  uint32_t *hub_base = nullptr;      // their first chunk number (ascending)
  uint32_t *dead = nullptr;          // vertices with out-degree 0 (teleport mode)
  uint32_t n_dead = 0;
  bool dead_dirty = true;
  double D_ref = 0.0;                // dead-end mass of the ranks under the graph they were computed on
  long long D_ref_n = 0;             // the same in 2^-62 units (64-bit mode)

  uint32_t *pend_src = nullptr, *pend_tgt = nullptr;  // pending marks of applied batches
  uint32_t pend_cap = 0;
  uint32_t n_pend_src = 0, n_pend_tgt = 0;
  bool pend_all = false;

  RankCtl *ctl = nullptr;            // device
  RankCtl *ctl_h = nullptr;          // pinned host mirror
  DeadPart *dpart = nullptr;         // [2][rank_grid]
  int rank_grid = 0;                 // cooperative grid of the rank kernel
  int rank_grid_max = 0;             // most blocks that can be co-resident
  // CUDA-graph launch of rank calls (pr_set_graph_launch): captured once, kernel arguments
  // updated in place before every replay
  bool use_graph = false;
  cudaGraph_t cg = nullptr;
  cudaGraphExec_t cg_exec = nullptr;
  cudaGraphNode_t cg_kernel = nullptr;
  bool cg_f32 = false;
  bool cg_df = false;
  uint32_t last_list_cnt[3] = {0, 0, 0};
  bool last_full = false;

  ApplyScratch sc;
  ApplyCtl *actl = nullptr, *actl_h = nullptr;
  uint32_t *big = nullptr;           // scratch for rows longer than shared memory
  uint64_t big_cap = 0;
  uint32_t *gen_tmp = nullptr;       // general scratch (scans, flags) sized n + 8
  uint32_t *gen_tmp2 = nullptr;
  uint32_t *scan_tmp = nullptr;      // block sums of scans over n
  double ms_apply = 0.0;
  // batched form: ncomp independent graphs; graph c owns vertices [comp_first[c], comp_first[c+1])
  uint32_t ncomp = 1;
  std::vector<uint32_t> comp_first;
  uint16_t *comp = nullptr;          // [n] graph of each vertex (ncomp > 1)
  void *comp_base = nullptr;         // [ncomp] (1 - alpha) / n_c, rank representation
  void *comp_init = nullptr;         // [ncomp] 1 / n_c
  unsigned long long *dRc = nullptr; // [3][ncomp]
  uint32_t *comp_out = nullptr;      // [ncomp][4]
  unsigned long long *comp_last = nullptr;
  std::vector<pr_stats> comp_stats;  // per graph, from the last rank call
  uint32_t dense_div = 16;           // dense iterations once affected > n / dense_div
  bool split_df = true;              // dense iterations of marking calls continue in per-iteration launches
  int32_t barrier_us = 0;            // grid-barrier wait limit of the persistent launches (0 = 4 s)
  uint32_t chunk_len = kChunk;       // sweep order: edges per chunk of a tier-2 row (128, 256 or 512)
  uint32_t group_max = kGroupMax;    // sweep order: longest row of an 8-lane group (16, 32 or 64)
  std::vector<double> trace_ms;      // last rank call: phase 0, then each iteration (device clock)
  std::vector<int64_t> trace_aff;    // affected vertices at the start of each iteration
  std::vector<int32_t> trace_kind;   // 0 sparse, 1 dense, 2 dense after compaction, 3 all vertices
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // per-iteration sweep launches (sweep.cu): change flags of the dense Dynamic Frontier
  // iterations and the CUDA graphs that loop over the iterations on the device
  uint8_t *emap = nullptr;           // [2][n] rank change above tau_f, by iteration parity; 0 between calls
  void *loops = nullptr;             // sweep.cu's cached graphs
  int sweep_grid = 0;                // blocks of a full-sweep launch
  int dfsweep_grid = 0;              // blocks of an all-item dense Dynamic Frontier sweep launch
  int cmpsweep_grid = 0;             // blocks of a compacted dense Dynamic Frontier sweep launch
  int pro_grid = 0;                  // blocks of the cooperative prologue launch
  bool loop_sweeps = true;           // single-graph self-loop handles iterate in per-iteration launches
  std::string err;
};

// graph.cu
pr_status graph_build(Graph *g, uint64_t m_in, const uint32_t *src_d, const uint32_t *dst_d);
// Applies nb batches in sequence (nb = 1: one batch).  off_d = device copy of the del and
// ins offsets ([nb + 1] each, del first), or null for a single batch.
pr_status graph_apply(Graph *g, uint64_t nd, const uint32_t *ds_d, const uint32_t *dd_d, uint64_t ni,
                      const uint32_t *is_d, const uint32_t *id_d, int nb, const uint32_t *off_d);
pr_status apply_scratch(Graph *g, uint64_t N);
constexpr int kOrderFromMax = 0, kOrderFromSeeds = 1, kOrderPerGraph = 2;
pr_status vertex_order(Graph *g, int kind, uint32_t *perm, uint32_t *inv,
                       const std::vector<uint32_t> *comp_n = nullptr);
pr_status order_cost(Graph *g, const uint32_t *perm, const uint32_t *inv, uint64_t cost[2]);  // order.cu, on a built graph
void map_ids(const uint32_t *inv, uint32_t *a, uint64_t m, cudaStream_t st);
pr_status graph_export(Graph *g, int dir, uint64_t *offs_h, uint32_t *cols_h);
pr_status graph_refresh_ident(Graph *g);
pr_status graph_refresh_dead(Graph *g);
void graph_free(Graph *g);
pr_status cuda_fail(Graph *g, cudaError_t e, const char *what);

// rank.cu
enum RankMode { kModeDF = 0, kModeNaive = 1, kModeStatic = 2, kModeDT = 3, kModeDFAsync = 4 };
pr_status rank_setup(Graph *g);  // grid size, control block
pr_status rank_run(Graph *g, RankMode mode, pr_stats *stats);
pr_status rank_init_contrib(Graph *g);  // C = R * adeg for all v, both parities
pr_status rank_check(Graph *g, const double *in_d);  // PR_ERR_INVALID_ARG unless finite, in [0, 2], sum <= 2
pr_status rank_set(Graph *g, const double *in_d);
pr_status rank_get(Graph *g, double *out_d);
pr_status rank_dead_mass(Graph *g, double *D);
pr_status components_setup(Graph *g, const std::vector<uint32_t> &comp_n);  // after graph_build

// sweep.cu: Static / Naive-dynamic iterations, and the dense iterations of a Dynamic
// Frontier, Dynamic Traversal or asynchronous call, one launch per iteration inside a
// CUDA-graph loop whose condition the last block of each sweep sets on the device.
pr_status sweep_setup(Graph *g);
bool sweep_eligible(const Graph *g);  // single graph, self-loop mode, no graph-launch mode
pr_status sweep_full(Graph *g, bool from_init);                  // all vertices, every iteration
pr_status sweep_dense(Graph *g, RankMode mode, const void *rank_args);  // after the marking launch's handoff
void sweep_free(Graph *g);

}  // namespace prdf

// The opaque handle of the C ABI.
struct pr_graph {
  prdf::Graph g;
  double *stage = nullptr;  // n doubles for host <-> device rank copies
};

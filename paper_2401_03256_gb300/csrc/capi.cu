// capi.cu - the extern "C" entry points declared in include/prdf.h.
//
// Validation happens here, before any device state is touched, so that a rejected call
// leaves the graph and its ranks as they were.  Host arrays are copied to the device;
// device arrays are used in place.
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "prdf_graph.cuh"


namespace {

thread_local std::string g_create_err;

// Makes the handle's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool is_device_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

pr_status invalid(prdf::Graph *g, const char *msg) {
  if (g) g->err = msg; else g_create_err = msg;
  return PR_ERR_INVALID_ARG;
}

pr_status check_params(const pr_params &p, std::string *why) {
  if (!(p.alpha > 0.0 && p.alpha < 1.0)) { *why = "alpha must be in (0, 1)"; return PR_ERR_INVALID_ARG; }
  if (!(p.tol >= 0.0) || !(p.frontier_tol >= 0.0) || std::isnan(p.tol) || std::isnan(p.frontier_tol)) {
    *why = "tolerances must be >= 0";
    return PR_ERR_INVALID_ARG;
  }
  if (p.max_iter < 0 || p.max_iter > prdf::kMaxIterLimit) { *why = "max_iter must be in [0, 1000]"; return PR_ERR_INVALID_ARG; }
  if (p.precision != PR_F64 && p.precision != PR_F32) { *why = "unknown precision"; return PR_ERR_INVALID_ARG; }
  if (p.dead_end != PR_DEADEND_SELFLOOP && p.dead_end != PR_DEADEND_TELEPORT) { *why = "unknown dead-end mode"; return PR_ERR_INVALID_ARG; }
  if (p.bin_lo < 0 || p.bin_hi < 0 || p.bin_hi < p.bin_lo) { *why = "need 0 <= bin_lo <= bin_hi"; return PR_ERR_INVALID_ARG; }
  if (p.vertex_order < 0 || p.vertex_order > 3) { *why = "vertex_order must be 0, 1, 2 or 3"; return PR_ERR_INVALID_ARG; }
  return PR_OK;
}

}  // namespace

using prdf::Graph;

namespace prdf {
static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(unsigned long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
static std::atomic<long long> g_alloc_left{-1};  // allocations that still succeed (-1: no injection)
bool alloc_fault() {
  long long left = g_alloc_left.load(std::memory_order_relaxed);
  while (left > 0 && !g_alloc_left.compare_exchange_weak(left, left - 1, std::memory_order_relaxed)) {
  }
  return left == 0;
}
}  // namespace prdf

extern "C" {

static pr_status ensure_stage(pr_graph *h);

void pr_params_default(pr_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->alpha = 0.85;
  p->tol = 1e-10;
  p->frontier_tol = p->tol / 1e5;
  p->max_iter = 500;
  p->precision = PR_F64;
  p->dead_end = PR_DEADEND_SELFLOOP;
  p->bin_lo = 8;
  p->bin_hi = 4096;
  p->vertex_order = 0;
}

const char *pr_status_string(pr_status s) {
  switch (s) {
    case PR_OK: return "PR_OK";
    case PR_ERR_INVALID_ARG: return "PR_ERR_INVALID_ARG";
    case PR_ERR_VERTEX_RANGE: return "PR_ERR_VERTEX_RANGE";
    case PR_ERR_OUT_OF_MEMORY: return "PR_ERR_OUT_OF_MEMORY";
    case PR_ERR_CUDA: return "PR_ERR_CUDA";
    case PR_ERR_DEVICE_TIMEOUT: return "PR_ERR_DEVICE_TIMEOUT";
    case PR_ERR_CAPACITY: return "PR_ERR_CAPACITY";
  }
  return "unknown status";
}

pr_status pr_get_trace(const pr_graph *h, int32_t cap, double *phase_ms, double *iter_ms, int64_t *affected,
                       int32_t *kind, int32_t *count) {
  if (!h) return invalid(nullptr, "graph is NULL");
  const Graph &g = h->g;
  if (cap < 0) return PR_ERR_INVALID_ARG;
  const int32_t k = g.trace_ms.empty() ? 0 : (int32_t)g.trace_ms.size() - 1;
  if (count) *count = k;
  if (phase_ms) *phase_ms = g.trace_ms.empty() ? 0.0 : g.trace_ms[0];
  for (int32_t i = 0; i < k && i < cap; i++) {
    if (iter_ms) iter_ms[i] = g.trace_ms[i + 1];
    if (affected) affected[i] = g.trace_aff[i];
    if (kind) kind[i] = g.trace_kind[i];
  }
  return PR_OK;
}

uint64_t pr_kernel_launches(void) { return prdf::g_launches.load(std::memory_order_relaxed); }

void pr_inject_alloc_failure(int32_t after) {
  prdf::g_alloc_left.store(after < 0 ? -1 : (long long)after, std::memory_order_relaxed);
}

const char *pr_last_error(const pr_graph *h) { return h ? h->g.err.c_str() : g_create_err.c_str(); }

static pr_status create_impl(uint32_t n, int64_t m, const uint32_t *src, const uint32_t *dst, const pr_params *params,
                             void *cuda_stream, const std::vector<uint32_t> *comp_n, pr_graph **out);

pr_status pr_graph_create(uint32_t n, int64_t m, const uint32_t *src, const uint32_t *dst, const pr_params *params,
                          void *cuda_stream, pr_graph **out) {
  return create_impl(n, m, src, dst, params, cuda_stream, nullptr, out);
}

pr_status pr_graph_create_batched(int32_t ncomp, const uint32_t *comp_n, int64_t m, const uint32_t *src,
                                  const uint32_t *dst, const pr_params *params, void *cuda_stream, pr_graph **out) {
  if (!out) return invalid(nullptr, "out is NULL");
  *out = nullptr;
  if (ncomp < 1 || ncomp > (int32_t)prdf::kMaxComponents || !comp_n)
    return invalid(nullptr, "ncomp must be in [1, 1024] with comp_n given");
  std::vector<uint32_t> cn(comp_n, comp_n + ncomp);
  uint64_t total = 0;
  for (uint32_t x : cn) {
    if (x == 0) return invalid(nullptr, "every graph needs at least one vertex");
    total += x;
  }
  if (total > 0xFFFFFFFFull) return invalid(nullptr, "more than 2^32 - 1 vertices in all");
  pr_params p;
  if (params) p = *params; else pr_params_default(&p);
  if (p.dead_end == PR_DEADEND_TELEPORT && ncomp > 1)
    return invalid(nullptr, "batched handles use self-loops for dead ends");
  return create_impl((uint32_t)total, m, src, dst, &p, cuda_stream, ncomp > 1 ? &cn : nullptr, out);
}

pr_status pr_get_component_stats(const pr_graph *h, pr_stats *stats, int32_t ncomp) {
  if (!h) return invalid(nullptr, "graph is NULL");
  if (!stats || ncomp != (int32_t)h->g.ncomp) return PR_ERR_INVALID_ARG;
  if (h->g.ncomp == 1) return PR_ERR_INVALID_ARG;
  for (int32_t c = 0; c < ncomp; c++) stats[c] = h->g.comp_stats[c];
  return PR_OK;
}

pr_status pr_set_tuning(pr_graph *h, const pr_tuning *t) {
  if (!h) return invalid(nullptr, "graph is NULL");
  Graph &g = h->g;
  if (!t || t->bin_lo < 1 || t->bin_hi < t->bin_lo || t->dense_div < 1 || t->blocks_per_sm < 1 ||
      t->blocks_per_sm * g.sm_count > g.rank_grid_max || (t->df_split != 0 && t->df_split != 1) || t->barrier_us < 0 ||
      t->chunk_len < 32 || t->chunk_len > (int32_t)prdf::kChunk || t->chunk_len % 32 != 0 || t->group_max < 0 ||
      t->group_max > (int32_t)prdf::kGroupMax)
    return invalid(&g, "need 1 <= bin_lo <= bin_hi, dense_div >= 1, blocks_per_sm within the resident limit, "
                       "barrier_us >= 0, chunk_len a multiple of 32 in [32, 512], group_max in [0, 64]");
  DeviceGuard dg(g.device);
  pr_tuning old;
  pr_get_tuning(h, &old);
  auto store = [&g](const pr_tuning &u) {
    if (u.bin_lo != g.p.bin_lo || (uint32_t)u.chunk_len != g.chunk_len || (uint32_t)u.group_max != g.group_max)
      g.ident_dirty = true;
    g.chunk_len = (uint32_t)u.chunk_len;
    g.group_max = (uint32_t)u.group_max;
    g.p.bin_lo = u.bin_lo;
    g.p.bin_hi = u.bin_hi;
    g.dense_div = (uint32_t)u.dense_div;
    g.rank_grid = u.blocks_per_sm * g.sm_count;
    g.split_df = u.df_split != 0;
    g.barrier_us = u.barrier_us;
  };
  store(*t);
  pr_status rc = prdf::graph_refresh_ident(&g);
  if (rc == PR_ERR_CAPACITY) {  // a tile this graph does not fit: keep the previous tuning
    const std::string why = g.err;
    store(old);
    pr_status r2 = prdf::graph_refresh_ident(&g);
    g.err = why;
    if (r2 != PR_OK) return r2;
  }
  return rc;
}

pr_status pr_get_tuning(const pr_graph *h, pr_tuning *t) {
  if (!h || !t) return invalid(nullptr, "NULL argument");
  const Graph &g = h->g;
  t->bin_lo = g.p.bin_lo;
  t->bin_hi = g.p.bin_hi;
  t->dense_div = (int32_t)g.dense_div;
  t->blocks_per_sm = g.rank_grid / g.sm_count;
  t->df_split = g.split_df ? 1 : 0;
  t->barrier_us = g.barrier_us;
  t->chunk_len = (int32_t)g.chunk_len;
  t->group_max = (int32_t)g.group_max;
  t->ms = 0.0;
  return PR_OK;
}

pr_status pr_set_graph_launch(pr_graph *h, int32_t enable) {
  if (!h) return invalid(nullptr, "graph is NULL");
  h->g.use_graph = enable != 0;
  return PR_OK;
}

// Autotuner: times Naive-dynamic sweeps of sweep_iters iterations (the full-sweep cost the
// thresholds steer) for every candidate bin_lo x blocks-per-SM, then, at the fastest of
// those, every sweep tile (chunk_len x group_max); keeps the fastest and restores the ranks.
// FP64 results do not depend on the choice; FP32 ones only through the order of additions.
pr_status pr_autotune(pr_graph *h, int32_t sweep_iters, pr_tuning *chosen) {
  if (!h) return invalid(nullptr, "graph is NULL");
  Graph &g = h->g;
  if (sweep_iters < 1 || sweep_iters > 100) return invalid(&g, "sweep_iters must be in [1, 100]");
  DeviceGuard dg(g.device);
  pr_status rc = ensure_stage(h);
  if (rc != PR_OK) return rc;
  if ((rc = prdf::rank_get(&g, h->stage)) != PR_OK) return rc;
  const int32_t keep_iter = g.p.max_iter;
  const uint32_t keep_pend_src = g.n_pend_src, keep_pend_tgt = g.n_pend_tgt;
  const bool keep_all = g.pend_all;
  const double keep_apply = g.ms_apply;
  pr_tuning cur{};
  pr_get_tuning(h, &cur);
  pr_tuning best = cur;
  best.ms = 1e30;
  const int32_t los[] = {4, 8, 16, 32};
  const int per_sm_max = std::max(1, g.rank_grid_max / g.sm_count);
  g.p.max_iter = sweep_iters;
  // time candidate t (best of two); a capacity refusal of a tile only skips that tile
  auto trial = [&](const pr_tuning &t) -> pr_status {
    pr_status r = pr_set_tuning(h, &t);
    if (r == PR_ERR_CAPACITY) return PR_OK;
    if (r != PR_OK) return r;
    pr_stats st;
    double ms = 1e30;
    for (int rep = 0; rep < 2 && r == PR_OK; rep++) {
      g.n_pend_src = 0;
      g.n_pend_tgt = 0;
      if ((r = prdf::rank_run(&g, prdf::kModeNaive, &st)) == PR_OK) ms = std::min(ms, st.ms_rank);
      if (r == PR_OK) r = prdf::rank_set(&g, h->stage);
    }
    if (r == PR_OK && ms < best.ms) {
      best = t;
      best.ms = ms;
    }
    return r;
  };
  for (int32_t lo : los) {
    for (int bps = std::max(1, per_sm_max - 2); bps <= per_sm_max && rc == PR_OK; bps++) {
      pr_tuning t = cur;
      t.bin_lo = lo;
      t.bin_hi = std::max(cur.bin_hi, lo);
      t.blocks_per_sm = bps;
      rc = trial(t);
    }
    if (rc != PR_OK) break;
  }
  const int32_t chunks[] = {128, 256, 512}, groups[] = {16, 32, 64};
  const pr_tuning base = best;
  for (int32_t c : chunks) {
    for (int32_t gm : groups) {
      if (rc != PR_OK || (c == base.chunk_len && gm == base.group_max)) continue;
      pr_tuning t = base;
      t.chunk_len = c;
      t.group_max = gm;
      rc = trial(t);
    }
  }
  g.p.max_iter = keep_iter;
  g.n_pend_src = keep_pend_src;
  g.n_pend_tgt = keep_pend_tgt;
  g.pend_all = keep_all;
  g.ms_apply = keep_apply;
  if (rc != PR_OK) return rc;
  if ((rc = pr_set_tuning(h, &best)) != PR_OK) return rc;
  if ((rc = prdf::rank_set(&g, h->stage)) != PR_OK) return rc;
  if (chosen) *chosen = best;
  return PR_OK;
}

static pr_status create_impl(uint32_t n, int64_t m, const uint32_t *src, const uint32_t *dst, const pr_params *params,
                             void *cuda_stream, const std::vector<uint32_t> *comp_n, pr_graph **out) {
  if (!out) return invalid(nullptr, "out is NULL");
  *out = nullptr;
  if (n == 0) return invalid(nullptr, "n must be >= 1");
  if (m < 0 || (m > 0 && (!src || !dst))) return invalid(nullptr, "bad edge arrays");
  if ((uint64_t)m >= 0xFFFFFFFFull) {
    g_create_err = "more than 2^32 - 1 input pairs";
    return PR_ERR_CAPACITY;
  }
  pr_params p;
  if (params) p = *params; else pr_params_default(&p);
  if (p.bin_lo == 0 && p.bin_hi == 0) {
    p.bin_lo = 8;
    p.bin_hi = 4096;
  }
  std::string why;
  if (check_params(p, &why) != PR_OK) return invalid(nullptr, why.c_str());

  pr_graph *h = new (std::nothrow) pr_graph;
  if (!h) {
    g_create_err = "host allocation failed";
    return PR_ERR_OUT_OF_MEMORY;
  }
  Graph &g = h->g;
  g.n = n;
  g.p = p;
  g.f32 = p.precision == PR_F32;
  g.teleport = p.dead_end == PR_DEADEND_TELEPORT;
  g.st = (cudaStream_t)cuda_stream;
  pr_status rc = PR_OK;
  uint32_t *tmp = nullptr;
  do {
    cudaError_t e = cudaGetDevice(&g.device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g.sm_count, cudaDevAttrMultiProcessorCount, g.device);
    int coop = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, g.device);
    if (e != cudaSuccess) { rc = prdf::cuda_fail(&g, e, "device query"); break; }
    if (!coop) { g.err = "device does not support cooperative launch"; rc = PR_ERR_CUDA; break; }
    const uint32_t *sd = src, *dd = dst;
    // handles may number their vertices breadth-first (order.cu) unless asked not to (a
    // batched handle graph by graph, each within its id range); the edges are then
    // rewritten, so they need a device copy of their own
    if (comp_n && p.vertex_order == 3) {
      g.err = "vertex_order 3 is for single-graph handles";
      rc = PR_ERR_INVALID_ARG;
      break;
    }
    const bool reorder = p.vertex_order != 1 && m > 0;
    if (m > 0 && (reorder || !(is_device_ptr(src) && is_device_ptr(dst)))) {
      e = cudaMalloc((void **)&tmp, 8ull * (uint64_t)m);
      if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, src, 4ull * m, cudaMemcpyDefault, g.st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(tmp + m, dst, 4ull * m, cudaMemcpyDefault, g.st);
      if (e != cudaSuccess) { rc = prdf::cuda_fail(&g, e, "upload edges"); break; }
      sd = tmp;
      dd = tmp + m;
    }
    if (reorder) {
      // the numbering comes from a first build of the graph in the caller's numbering
      Graph g0;
      g0.n = n;
      g0.p = p;
      g0.f32 = g.f32;
      g0.teleport = g.teleport;
      g0.st = g.st;
      g0.device = g.device;
      g0.sm_count = g.sm_count;
      rc = prdf::graph_build(&g0, (uint64_t)m, sd, dd);
      // vertex_order 0: both numberings, the one with the cheaper modelled gathers kept if
      // it beats the caller's by 5%; 2 and 3: the one asked for, always
      const int kinds[2] = {comp_n ? prdf::kOrderPerGraph : prdf::kOrderFromMax, prdf::kOrderFromSeeds};
      uint32_t *cp[2] = {nullptr, nullptr}, *ci[2] = {nullptr, nullptr};
      uint64_t cost[2][2] = {{0, 0}, {0, 0}};
      int best = -1;
      for (int k = 0; k < 2 && rc == PR_OK; k++) {
        if ((p.vertex_order >= 2 && p.vertex_order - 2 != k) || (comp_n && k == 1)) continue;
        e = cudaMalloc((void **)&cp[k], 4ull * n);
        if (e == cudaSuccess) e = cudaMalloc((void **)&ci[k], 4ull * n);
        if (e != cudaSuccess) { rc = prdf::cuda_fail(&g0, e, "vertex numbering"); break; }
        rc = prdf::vertex_order(&g0, kinds[k], cp[k], ci[k], comp_n);
        if (rc == PR_OK && p.vertex_order == 0) rc = prdf::order_cost(&g0, cp[k], ci[k], cost[k]);
        if (rc == PR_OK && (best < 0 || cost[k][1] < cost[best][1])) best = k;
      }
      bool keep = rc == PR_OK && best >= 0 && (p.vertex_order >= 2 || cost[best][1] * 20 < cost[best][0] * 19);
      for (int k = 0; k < 2; k++) {
        if (keep && k == best) {
          g.perm = cp[k];
          g.inv = ci[k];
        } else {
          cudaFree(cp[k]);
          cudaFree(ci[k]);
        }
      }
      // no room for the numbering's transient build: the caller's numbering (vertex_order 0)
      const bool fallback = rc == PR_ERR_OUT_OF_MEMORY && p.vertex_order == 0;
      if (rc != PR_OK && !fallback) g.err = g0.err;
      prdf::graph_free(&g0);
      if (fallback) rc = PR_OK;
      if (rc != PR_OK) break;
      if (keep) {
        prdf::map_ids(g.inv, tmp, 2ull * (uint64_t)m, g.st);
        g.perm_h.resize(n);
        e = cudaMemcpyAsync(g.perm_h.data(), g.perm, 4ull * n, cudaMemcpyDeviceToHost, g.st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g.st);
        if (e != cudaSuccess) { rc = prdf::cuda_fail(&g, e, "vertex numbering"); break; }
      }
    }
    rc = prdf::graph_build(&g, (uint64_t)m, sd, dd);
    if (rc != PR_OK) break;
    if (comp_n && (rc = prdf::components_setup(&g, *comp_n)) != PR_OK) break;
    rc = prdf::rank_setup(&g);
  } while (0);
  if (tmp) {
    cudaStreamSynchronize(g.st);
    cudaFree(tmp);
  }
  if (rc != PR_OK) {
    g_create_err = g.err;
    prdf::graph_free(&g);
    delete h;
    return rc;
  }
  *out = h;
  return PR_OK;
}

pr_status pr_graph_destroy(pr_graph *h) {
  if (!h) return PR_OK;
  {
    DeviceGuard dg(h->g.device);
    cudaStreamSynchronize(h->g.st);
    prdf::graph_free(&h->g);
    cudaFree(h->stage);
  }
  delete h;
  return PR_OK;
}

// Shared by pr_apply_batch (nb = 1, no offsets) and pr_apply_batches.
static pr_status apply_impl(pr_graph *h, int32_t nb, const int64_t *del_off, const int64_t *ins_off, int64_t n_del,
                            const uint32_t *del_src, const uint32_t *del_dst, int64_t n_ins, const uint32_t *ins_src,
                            const uint32_t *ins_dst) {
  Graph &g = h->g;
  if ((n_del > 0 && (!del_src || !del_dst)) || (n_ins > 0 && (!ins_src || !ins_dst)))
    return invalid(&g, "batch array is NULL");
  const uint64_t N = (uint64_t)n_del + (uint64_t)n_ins;
  if (N == 0) return PR_OK;
  if (N > (1ull << 31)) return invalid(&g, "batch too large (more than 2^31 pairs)");
  DeviceGuard dg(g.device);
  const uint32_t *arr[4] = {del_src, del_dst, ins_src, ins_dst};
  const uint64_t len[4] = {(uint64_t)n_del, (uint64_t)n_del, (uint64_t)n_ins, (uint64_t)n_ins};
  // host arrays are checked here, before anything is copied or changed
  for (int k = 0; k < 4; k++) {
    if (!len[k] || is_device_ptr(arr[k])) continue;
    for (uint64_t i = 0; i < len[k]; i++)
      if (arr[k][i] >= g.n) {
        g.err = "vertex id out of range";
        return PR_ERR_VERTEX_RANGE;
      }
  }
  pr_status rc = prdf::apply_scratch(&g, N);
  if (rc != PR_OK) return rc;
  std::vector<uint32_t> off_h;
  if (nb > 1) {
    prdf::ApplyScratch &s = g.sc;
    if (nb > s.boff_cap) {
      cudaFree(s.boff);
      s.boff = nullptr;
      s.boff_cap = 0;
      cudaError_t e = cudaMalloc(&s.boff, sizeof(uint32_t) * 2 * ((uint64_t)nb + 1));
      if (e != cudaSuccess) return prdf::cuda_fail(&g, e, "batch offsets");
      s.boff_cap = nb;
    }
    off_h.resize(2 * ((size_t)nb + 1));
    for (int32_t k = 0; k <= nb; k++) {
      off_h[k] = (uint32_t)del_off[k];
      off_h[nb + 1 + k] = (uint32_t)ins_off[k];
    }
  }
  cudaError_t e = cudaEventRecord(g.ev0, g.st);
  if (e == cudaSuccess && nb > 1)
    e = cudaMemcpyAsync(g.sc.boff, off_h.data(), sizeof(uint32_t) * off_h.size(), cudaMemcpyHostToDevice, g.st);
  const uint32_t *dev[4];
  uint32_t *stage = g.sc.pairs;
  for (int k = 0; k < 4 && e == cudaSuccess; k++) {
    if (!len[k] || is_device_ptr(arr[k])) {
      dev[k] = arr[k];
    } else {
      e = cudaMemcpyAsync(stage, arr[k], 4ull * len[k], cudaMemcpyHostToDevice, g.st);
      dev[k] = stage;
    }
    stage += len[k];
  }
  if (e != cudaSuccess) return prdf::cuda_fail(&g, e, "upload batch");
  // graph_apply synchronises the stream before it returns, so off_h outlives its copy
  rc = prdf::graph_apply(&g, (uint64_t)n_del, dev[0], dev[1], (uint64_t)n_ins, dev[2], dev[3], nb > 1 ? nb : 1,
                         nb > 1 ? g.sc.boff : nullptr);
  if (rc != PR_OK) return rc;
  e = cudaEventRecord(g.ev1, g.st);
  if (e == cudaSuccess) e = cudaEventSynchronize(g.ev1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, g.ev0, g.ev1);
  if (e != cudaSuccess) return prdf::cuda_fail(&g, e, "apply timing");
  g.ms_apply += ms;
  return PR_OK;
}

pr_status pr_apply_batch(pr_graph *h, int64_t n_del, const uint32_t *del_src, const uint32_t *del_dst,
                         int64_t n_ins, const uint32_t *ins_src, const uint32_t *ins_dst) {
  if (!h) return invalid(nullptr, "graph is NULL");
  if (n_del < 0 || n_ins < 0) return invalid(&h->g, "negative batch size");
  return apply_impl(h, 1, nullptr, nullptr, n_del, del_src, del_dst, n_ins, ins_src, ins_dst);
}

pr_status pr_apply_batches(pr_graph *h, int32_t n_batches, const int64_t *del_off, const uint32_t *del_src,
                           const uint32_t *del_dst, const int64_t *ins_off, const uint32_t *ins_src,
                           const uint32_t *ins_dst) {
  if (!h) return invalid(nullptr, "graph is NULL");
  Graph &g = h->g;
  if (n_batches < 0 || n_batches > PR_MAX_BATCHES) return invalid(&g, "batch count out of range");
  if (n_batches == 0) return PR_OK;
  if (!del_off || !ins_off) return invalid(&g, "offset array is NULL");
  if (del_off[0] != 0 || ins_off[0] != 0) return invalid(&g, "offsets must start at 0");
  for (int32_t k = 0; k < n_batches; k++)
    if (del_off[k + 1] < del_off[k] || ins_off[k + 1] < ins_off[k]) return invalid(&g, "offsets must not decrease");
  if (del_off[n_batches] + ins_off[n_batches] > (int64_t)(1ull << 31))
    return invalid(&g, "batch too large (more than 2^31 pairs)");
  return apply_impl(h, n_batches, del_off, ins_off, del_off[n_batches], del_src, del_dst, ins_off[n_batches], ins_src,
                    ins_dst);
}

static pr_status run(pr_graph *h, prdf::RankMode mode, pr_stats *stats) {
  if (!h) return invalid(nullptr, "graph is NULL");
  DeviceGuard dg(h->g.device);
  if (stats) std::memset(stats, 0, sizeof(*stats));
  return prdf::rank_run(&h->g, mode, stats);
}

pr_status pr_static(pr_graph *h, pr_stats *stats) { return run(h, prdf::kModeStatic, stats); }
pr_status pr_naive_dynamic(pr_graph *h, pr_stats *stats) { return run(h, prdf::kModeNaive, stats); }
pr_status pr_dynamic_frontier(pr_graph *h, pr_stats *stats) { return run(h, prdf::kModeDF, stats); }
pr_status pr_dynamic_traversal(pr_graph *h, pr_stats *stats) { return run(h, prdf::kModeDT, stats); }
pr_status pr_dynamic_frontier_async(pr_graph *h, pr_stats *stats) { return run(h, prdf::kModeDFAsync, stats); }

static pr_status ensure_stage(pr_graph *h) {
  if (h->stage) return PR_OK;
  cudaError_t e = cudaMalloc((void **)&h->stage, sizeof(double) * h->g.n);
  if (e != cudaSuccess) return prdf::cuda_fail(&h->g, e, "rank staging buffer");
  return PR_OK;
}

pr_status pr_get_ranks(pr_graph *h, double *out, uint32_t n) {
  if (!h) return invalid(nullptr, "graph is NULL");
  Graph &g = h->g;
  if (!out || n != g.n) return invalid(&g, "out must hold exactly n doubles");
  DeviceGuard dg(g.device);
  pr_status rc;
  cudaError_t e;
  if (is_device_ptr(out)) {
    if ((rc = prdf::rank_get(&g, out)) != PR_OK) return rc;
    e = cudaStreamSynchronize(g.st);
  } else {
    if ((rc = ensure_stage(h)) != PR_OK) return rc;
    if ((rc = prdf::rank_get(&g, h->stage)) != PR_OK) return rc;
    e = cudaMemcpyAsync(out, h->stage, sizeof(double) * n, cudaMemcpyDeviceToHost, g.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g.st);
  }
  if (e != cudaSuccess) return prdf::cuda_fail(&g, e, "get ranks");
  return PR_OK;
}

pr_status pr_set_ranks(pr_graph *h, const double *in, uint32_t n) {
  if (!h) return invalid(nullptr, "graph is NULL");
  Graph &g = h->g;
  if (!in || n != g.n) return invalid(&g, "in must hold exactly n doubles");
  DeviceGuard dg(g.device);
  pr_status rc;
  if (is_device_ptr(in)) {
    if ((rc = prdf::rank_check(&g, in)) != PR_OK) return rc;
    return prdf::rank_set(&g, in);
  }
  if ((rc = ensure_stage(h)) != PR_OK) return rc;
  cudaError_t e = cudaMemcpyAsync(h->stage, in, sizeof(double) * n, cudaMemcpyHostToDevice, g.st);
  if (e != cudaSuccess) return prdf::cuda_fail(&g, e, "set ranks");
  if ((rc = prdf::rank_check(&g, h->stage)) != PR_OK) return rc;
  return prdf::rank_set(&g, h->stage);
}

pr_status pr_graph_info(const pr_graph *h, uint32_t *n, int64_t *m) {
  if (!h) return invalid(nullptr, "graph is NULL");
  if (n) *n = h->g.n;
  if (m) *m = (int64_t)h->g.m;
  return PR_OK;
}

pr_status pr_get_csr(pr_graph *h, int32_t dir, uint64_t *offs, uint32_t *cols) {
  if (!h) return invalid(nullptr, "graph is NULL");
  Graph &g = h->g;
  if ((dir != 0 && dir != 1) || !offs || (!cols && g.m > 0)) return invalid(&g, "bad arguments");
  DeviceGuard dg(g.device);
  return prdf::graph_export(&g, dir, offs, cols);
}

pr_status pr_get_affected(pr_graph *h, uint32_t *out, int64_t cap, int64_t *count) {
  if (!h) return invalid(nullptr, "graph is NULL");
  Graph &g = h->g;
  if (!count || cap < 0 || (cap > 0 && !out)) return invalid(&g, "bad arguments");
  DeviceGuard dg(g.device);
  if (g.last_full) {
    *count = g.n;
    for (int64_t i = 0; i < cap && i < (int64_t)g.n; i++) out[i] = (uint32_t)i;
    return PR_OK;
  }
  int64_t total = 0;
  for (int b = 0; b < 3; b++) {
    int64_t c = g.last_list_cnt[b];
    int64_t take = std::max<int64_t>(0, std::min<int64_t>(c, cap - total));
    if (take > 0) {
      cudaError_t e = cudaMemcpyAsync(out + total, g.list[b], 4ull * take, cudaMemcpyDeviceToHost, g.st);
      if (e != cudaSuccess) return prdf::cuda_fail(&g, e, "get affected");
    }
    total += c;
  }
  cudaError_t e = cudaStreamSynchronize(g.st);
  if (e != cudaSuccess) return prdf::cuda_fail(&g, e, "get affected");
  if (!g.perm_h.empty())  // back to the caller's numbering
    for (int64_t i = 0; i < std::min<int64_t>(total, cap); i++) out[i] = g.perm_h[out[i]];
  *count = total;
  return PR_OK;
}

}  // extern "C"

/*
 * prdf.h - C ABI of the GB300 (sm_103a) Dynamic Frontier PageRank library (libprdf.so).
 *
 * The method is S. Sahu, "An Incrementally Expanding Approach for Updating PageRank on
 * Dynamic Graphs" (arXiv 2401.03256).  A graph lives on one GPU behind an opaque handle;
 * a batch of edge deletions and insertions is applied to it, and the ranks are brought
 * up to date by Static, Naive-dynamic or Dynamic Frontier PageRank.
 *
 * Conventions for every entry point:
 *  - Vertex ids are uint32 in [0, n) (Section 5.1.2: 32-bit vertex ids).
 *  - Array arguments may be host or device pointers; the library finds out which with
 *    cudaPointerGetAttributes and copies as needed.  The caller keeps ownership of
 *    every array it passes; nothing is retained after the call returns.
 *  - The handle owns all device memory it allocates until pr_graph_destroy.
 *  - All device work of a handle runs on the stream given at creation (NULL = the
 *    legacy default stream).  Every call returns after that work has finished.
 *  - Errors: every call returns a pr_status.  Arguments are validated before anything
 *    is changed, so on PR_ERR_INVALID_ARG / PR_ERR_VERTEX_RANGE the graph and its
 *    ranks are as before the call.  pr_last_error gives a one-line message.
 *  - One writer per handle (Section 3.2: one writer on the graph at a time).  Calls on
 *    the same handle must not overlap; different handles are independent.
 *  - Not converging within max_iter is not an error: the call returns PR_OK with
 *    stats.converged = 0 (Algorithm 1 returns its ranks at MAX_ITERATIONS).
 */
#ifndef PRDF_H
#define PRDF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pr_graph pr_graph; /* opaque handle */

typedef enum {
    PR_OK = 0,
    PR_ERR_INVALID_ARG = 1,    /* bad parameter, size or NULL pointer */
    PR_ERR_VERTEX_RANGE = 2,   /* a vertex id >= n */
    PR_ERR_OUT_OF_MEMORY = 3,  /* device allocation failed; the handle is unchanged */
    PR_ERR_CUDA = 4,           /* a CUDA runtime call failed (message in pr_last_error) */
    PR_ERR_DEVICE_TIMEOUT = 5, /* a bounded device-side wait (a grid barrier, or a staged copy
                                  into shared memory) gave up; ranks are undefined */
    PR_ERR_CAPACITY = 6        /* a size limit: more than 2^32 - 1 stored edges, a row needing
                                  more than 2^21 sweep chunks, or pr_static_noalloc's vertex cap */
} pr_status;

/* Rank arithmetic.  The paper computes in FP64 (Section 5.1.2); its tests are absolute
 * (L-inf change <= tau = 1e-10 stops, a change > tau_f = 1e-15 marks).
 *  PR_F64: 64-bit fixed point.  Ranks and contributions are int64 counts of 2^-62 (about
 *    2.2e-19); ranks enter as doubles rounded to the nearest unit and leave as the nearest
 *    double.  In-edge sums, the L-inf maximum and the dead-end mass are exact integer
 *    operations (so results do not depend on the order of the sums); each contribution
 *    alpha R[u] / |out(u)| is rounded once.  One sweep of Eq. 1 is therefore off the exact
 *    sweep of the same input by at most 2^-62 per in-edge of a vertex, and a whole call
 *    accumulates at most m * 2^-62 / (1 - alpha) in the L1 norm (m = stored edges), which
 *    bounds the L-inf error as well (7e-11 for m = 5e7; observed differences to FP64 are
 *    near 1e-17).  The resolution is absolute: a rank near 1/n keeps about 62 - log2(n)
 *    significant bits (40 at n = 2^22, 34 at n = 2^28), against 53 for an IEEE double.
 *    Values must stay below 2; pr_set_ranks enforces a distribution (sum <= 1), under
 *    which no rank or in-edge sum can reach that.
 *  PR_F32: IEEE single precision for ranks and contributions (half the bytes per gathered
 *    contribution); the L-inf test compares the float changes widened to double; in
 *    teleport mode the dead-end mass is summed in FP64 with Neumaier compensation. */
typedef enum { PR_F64 = 0, PR_F32 = 1 } pr_precision;

/* Dead ends (Section 3.1): the paper adds a self-loop to every vertex so no vertex has
 * out-degree 0.  PR_DEADEND_TELEPORT adds none and spreads a dead end's rank over all
 * vertices instead (the "global teleport contribution" the paper avoids). */
typedef enum { PR_DEADEND_SELFLOOP = 0, PR_DEADEND_TELEPORT = 1 } pr_deadend;

typedef struct {
    double alpha;         /* damping factor; 0.85 (Section 5.1.2) */
    double tol;           /* iteration tolerance tau on the L-inf norm; 1e-10 (Section 5.1.2) */
    double frontier_tol;  /* frontier tolerance tau_f; tau / 1e5 (Section 4.3) */
    int32_t max_iter;     /* MAX_ITERATIONS; 500 (Section 5.1.2); at most 1000 */
    int32_t precision;    /* pr_precision: rank arithmetic (64-bit fixed point or FP32) */
    int32_t dead_end;     /* pr_deadend */
    int32_t bin_lo;       /* in-degree <= bin_lo: one thread per vertex (0 = default 8) */
    int32_t bin_hi;       /* in-degree >  bin_hi: one block per vertex (0 = default 4096) */
    int32_t vertex_order; /* Internal vertex numbering of a handle.  A breadth-first
                             numbering (at most 1024 levels; the vertices not reached keep
                             their relative order after them) puts the contributions that
                             warps gather side by side close together: from the vertex of
                             largest degree (2) or from max(8192, n / 2048) vertices evenly
                             spaced in the caller's numbering as the first level (3).
                             0 (default): both are computed at creation and the one whose
                             short-row gathers a model finds cheapest is kept if it touches
                             at least 5% fewer 32-byte sectors than the caller's numbering (a
                             grid numbered row by row keeps its own); 1: keep the caller's
                             numbering.  Batched handles number each graph within its own id
                             range, breadth-first from its vertex of largest degree (0: if
                             the model finds it cheaper; 2: always; 3: PR_ERR_INVALID_ARG).
                             Ids are translated at every call: results, ranks, affected sets
                             and the CSR export are in the caller's numbering (a renumbered
                             handle keeps 8 B per vertex of translation tables on the device
                             and 4 B on the host).  Computing a numbering takes a second,
                             transient build of the graph on the device; without room for it
                             the caller's numbering is kept (0) or creation fails with
                             PR_ERR_OUT_OF_MEMORY (2, 3).  Other values: PR_ERR_INVALID_ARG. */
} pr_params;

typedef struct {
    int32_t iterations;         /* iterations run (Algorithm 1's loop count) */
    int32_t converged;          /* 1 if the L-inf change fell to <= tol */
    int64_t affected_final;     /* vertices marked affected by the end (all n for sweeps) */
    int64_t vertices_processed; /* sum over iterations of vertices whose rank was computed */
    int64_t edges_processed;    /* sum over iterations of their in-edges */
    double bytes_algorithmic;   /* algorithmic bytes moved by the rank kernel */
    double last_delta;          /* L-inf change of the last iteration */
    double ms_apply;            /* device time of pr_apply_batch calls since the last rank call */
    double ms_rank;             /* device time of this call's rank computation */
} pr_stats;

/* Fills the paper's defaults: alpha 0.85, tol 1e-10, frontier_tol 1e-15, max_iter 500,
 * FP64, self-loops, default degree bins. */
void pr_params_default(pr_params *params);

/* Builds a graph on the current CUDA device from m pairs (src[i], dst[i]).
 * Duplicates are dropped, pairs with src == dst are dropped, and in self-loop mode a
 * self-loop is added to every vertex (Section 3.1, Section 5.1.4).  Both adjacencies
 * (in-edges for the pull computation of Eq. 1, out-edges for the frontier marking of
 * Algorithm 1) are stored with each row sorted.  Ranks start at 1/n.
 * n >= 1; m >= 0; src/dst may be NULL when m == 0; params may be NULL for defaults;
 * cuda_stream is a cudaStream_t or NULL.  *out receives the handle. */
pr_status pr_graph_create(uint32_t n, int64_t m, const uint32_t *src, const uint32_t *dst,
                          const pr_params *params, void *cuda_stream, pr_graph **out);

/* Batched form: ncomp (1..1024) independent graphs in one handle, updated together.
 * Vertex ids are global: graph c owns [first_c, first_c + comp_n[c]) with
 * first_c = comp_n[0] + ... + comp_n[c-1] (each comp_n[c] >= 1).  src/dst hold the edges of
 * all graphs in global ids; an edge (or later a batch pair) joining two graphs is rejected
 * with PR_ERR_INVALID_ARG.  pr_apply_batch takes one combined batch for all graphs, and each
 * rank call runs every graph in one persistent launch: graph c uses its own (1 - alpha)/n_c
 * and starting rank 1/n_c (Eq. 1 per graph) and its own convergence test, and stops
 * updating once converged, so its ranks are those of a run of graph c alone.  Self-loop
 * dead-end mode only.  Per-graph results: pr_get_component_stats. */
pr_status pr_graph_create_batched(int32_t ncomp, const uint32_t *comp_n, int64_t m, const uint32_t *src,
                                  const uint32_t *dst, const pr_params *params, void *cuda_stream, pr_graph **out);

/* Per-graph statistics of the last rank call of a batched handle (ncomp entries, host):
 * iterations, converged, affected_final, last_delta; ms_rank is the whole launch. */
pr_status pr_get_component_stats(const pr_graph *g, pr_stats *stats, int32_t ncomp);

/* Work distribution of the rank kernels: in-degree thresholds of the thread and block bins
 * (bin_lo also bounds the rows a sweep gives one thread each), the dense-iteration divisor (an iteration sweeps the
 * compacted affected set once it exceeds n / dense_div vertices), the resident blocks per
 * SM of the persistent launch, and df_split (1, the default: a Dynamic Frontier, Dynamic
 * Traversal or asynchronous call on a single-graph handle in self-loop mode continues in
 * per-iteration launches once its affected set is dense (after its search for Dynamic
 * Traversal), growing the set by pulling marks from per-vertex change flags or pushing the
 * out-rows of first expansions; 0: everything in the one persistent launch), and the sweep
 * tiles: rows of bin_lo < in-degree <= max(bin_lo, group_max) take an 8-lane group each,
 * longer rows are cut into chunks of chunk_len in-edges taken by whole warps.  ms is the
 * time the autotuner measured (0 otherwise).  With PR_F64 results do not depend on any of
 * these (fixed-point sums are exact in any order); with PR_F32 a different tiling adds a
 * vertex's contributions in another order, which changes ranks by FP32 rounding only.
 * Defaults: bin_lo 8, bin_hi 4096, dense_div 16, chunk_len 512, group_max 64. */
typedef struct {
    int32_t bin_lo, bin_hi, dense_div, blocks_per_sm;
    int32_t df_split;
    int32_t barrier_us;  /* bounded wait of a grid barrier in the persistent launches, in
                            microseconds (0 = the default 4 s); a wait that runs out ends the
                            launch and the call returns PR_ERR_DEVICE_TIMEOUT.  A short value
                            exercises that path in tests. */
    int32_t chunk_len;   /* a multiple of 32 in [32, 512]; a vertex may have at most
                            2^21 chunks (else PR_ERR_CAPACITY) */
    int32_t group_max;   /* [0, 64] */
    double ms;
} pr_tuning;

/* Sets the tuning (rebuilds the degree-tiered sweep order if bin_lo changes). */
pr_status pr_set_tuning(pr_graph *g, const pr_tuning *t);
pr_status pr_get_tuning(const pr_graph *g, pr_tuning *t);

/* Autotuner: times sweep_iters-iteration Naive-dynamic sweeps of this graph for each
 * candidate bin_lo (4, 8, 16, 32) and blocks per SM, keeps the fastest, restores the ranks
 * and pending marks, and returns the choice in *chosen (may be NULL). */
pr_status pr_autotune(pr_graph *g, int32_t sweep_iters, pr_tuning *chosen);

/* enable != 0: rank calls replay one CUDA graph (control-block reset + the cooperative
 * persistent kernel), captured on first use; only the kernel's arguments change between
 * replays. */
pr_status pr_set_graph_launch(pr_graph *g, int32_t enable);

/* Fault injection on the host, for tests of the out-of-memory path: after this call the
 * next `after` allocations of graph storage and batch scratch (all handles, this process)
 * succeed and the following ones fail with PR_ERR_OUT_OF_MEMORY, as cudaMalloc failing
 * would; a negative `after` switches the injection off.  A failing call leaves the graph
 * as it was.  Never fails. */
void pr_inject_alloc_failure(int32_t after);

/* Frees all device memory of the handle.  NULL is accepted. */
pr_status pr_graph_destroy(pr_graph *g);

/* Applies one batch update (Section 3.2): E^t = (E^{t-1} \ D) U I, D = the n_del
 * deletions, I = the n_ins insertions.  Pairs with src == dst, deletions of absent edges,
 * insertions of present edges and duplicates have no effect; an edge both deleted and
 * inserted is present afterwards.  The effective changes Delta^- = E^{t-1} \ E^t and
 * Delta^+ = E^t \ E^{t-1} are remembered as pending marks for the next
 * pr_dynamic_frontier (they accumulate over several calls; any rank call consumes them).
 * Contributions of sources whose out-degree changed are refreshed. */
pr_status pr_apply_batch(pr_graph *g, int64_t n_del, const uint32_t *del_src, const uint32_t *del_dst,
                         int64_t n_ins, const uint32_t *ins_src, const uint32_t *ins_dst);

#define PR_MAX_BATCHES 65536

/* Applies n_batches batch updates one after another (Section 3.2 applied per batch) in one
 * pass: the graph afterwards is exactly the one that n_batches pr_apply_batch calls would
 * give.  Batch k deletes the pairs del_src/del_dst[del_off[k] .. del_off[k+1]) and inserts
 * ins_src/ins_dst[ins_off[k] .. ins_off[k+1]); del_off and ins_off are host arrays of
 * n_batches + 1 non-decreasing entries starting at 0 (PR_ERR_INVALID_ARG otherwise, and
 * for n_batches > PR_MAX_BATCHES or more than 2^31 pairs in all).  Only the net change
 * between the graph before the first batch and after the last becomes pending marks: an
 * edge deleted by one batch and inserted again by a later one marks nothing.  Pair arrays
 * may be host or device memory. */
pr_status pr_apply_batches(pr_graph *g, int32_t n_batches, const int64_t *del_off, const uint32_t *del_src,
                           const uint32_t *del_dst, const int64_t *ins_off, const uint32_t *ins_src,
                           const uint32_t *ins_dst);

/* Static PageRank (Section 3.1, Eq. 1): ranks restart at 1/n; every vertex is updated
 * each iteration until the L-inf change is <= tol or max_iter iterations ran.
 * stats may be NULL. */
pr_status pr_static(pr_graph *g, pr_stats *stats);

/* Naive-dynamic PageRank (Section 3.3.1): as pr_static but starting from the current ranks. */
pr_status pr_naive_dynamic(pr_graph *g, pr_stats *stats);

/* Dynamic Frontier PageRank (Algorithm 1, synchronous form of Section 4.2): marks the
 * out-neighbours of every source of the pending changes (and the deleted targets, which
 * are G^{t-1}.out(u) \ G^t.out(u)), then iterates over affected vertices only; a vertex
 * whose rank changes by more than frontier_tol marks its out-neighbours, which join from
 * the next iteration.  Stops when the L-inf change is <= tol or after max_iter iterations. */
pr_status pr_dynamic_frontier(pr_graph *g, pr_stats *stats);

/* Dynamic Traversal (Section 3.3.2, the paper's third comparator): every vertex reachable
 * from a source of the pending changes in G^{t-1} or G^t is affected (breadth-first
 * search in G^t from the sources and the deleted targets, which reaches the same set;
 * searches deeper than 1000 levels take every vertex), then the affected vertices iterate
 * as in pr_dynamic_frontier with no further marking.  In teleport mode any change affects
 * every vertex.  Consumes the pending marks like pr_dynamic_frontier. */
pr_status pr_dynamic_traversal(pr_graph *g, pr_stats *stats);

/* Asynchronous Dynamic Frontier (Section 4.2, the form the paper runs on the CPU): as
 * pr_dynamic_frontier, but with one rank vector updated in place, so a vertex may read
 * in-neighbour ranks already updated in the same iteration.  Results depend on the order
 * in which the GPU's threads run (not bit-reproducible from run to run); every run stops
 * under the same L-inf test.  Needs a single-graph handle in self-loop mode without graph
 * launch (PR_ERR_INVALID_ARG otherwise). */
pr_status pr_dynamic_frontier_async(pr_graph *g, pr_stats *stats);

/* Copies the n ranks (widened to double in FP32 mode) into out (host or device). */
pr_status pr_get_ranks(pr_graph *g, double *out, uint32_t n);

/* Replaces the ranks with in[0..n) (host or device), e.g. to resume or to start every
 * implementation from the same previous ranks.  Pending marks are kept.  The ranks must be
 * a distribution up to drift: every value finite and in [0, 2], and their sum at most 2
 * (for a batched handle, the sum over each graph's vertices).  Exact methods keep the sum
 * at 1; Dynamic Frontier leaves vertices outside its affected set as they were, so chained
 * updates drift from 1 slightly.  Otherwise PR_ERR_INVALID_ARG and the ranks are
 * unchanged. */
pr_status pr_set_ranks(pr_graph *g, const double *in, uint32_t n);

/* Number of vertices and of stored edges (self-loops included). */
pr_status pr_graph_info(const pr_graph *g, uint32_t *n, int64_t *m);

/* Exports one adjacency in packed CSR form into host arrays: dir 0 = out-edges (rows by
 * source), 1 = in-edges (rows by target); offs has n + 1 entries, cols has m entries
 * (m from pr_graph_info); each row ascending. */
pr_status pr_get_csr(pr_graph *g, int32_t dir, uint64_t *offs, uint32_t *cols);

/* Vertices marked affected by the last Dynamic Frontier (synchronous or asynchronous) or
 * Dynamic Traversal call, in no particular order, into a host array of capacity cap;
 * *count receives the total number (n after a call that took every vertex). */
pr_status pr_get_affected(pr_graph *g, uint32_t *out, int64_t cap, int64_t *count);

/* Trace of the last rank call (any of the rank entry points), from the device
 * clock: phase_ms = initial marking (phase 0); for each iteration i < *count (at most cap
 * entries written): iter_ms[i] its duration, affected[i] the vertices affected after it,
 * kind[i]: in the persistent marking launch 0 = affected lists, 1 = compacted sweep items
 * reused, 2 = sweep items compacted in this iteration, 4 = all sweep items scanned, those
 * of vertices stamped later skipped; 3 = all vertices; in the per-iteration launches of a
 * split call 5 = compacted items, 6 = all items with the stamp check, 7 = all items, vertices
 * not yet affected joining by pull from the previous iteration's change flags, 8 = compacted
 * items rebuilt before the sweep.  Any of the output arrays may be NULL (host memory). */
pr_status pr_get_trace(const pr_graph *g, int32_t cap, double *phase_ms, double *iter_ms, int64_t *affected,
                       int32_t *kind, int32_t *count);

/* Number of CUDA kernels this library has launched in this process (all handles),
 * for accounting of device work.  Never fails. */
uint64_t pr_kernel_launches(void);

/* ------------------------------------------------------ allocation-free Static PageRank ----
 * The paper has no counterpart to this entry point; it exists for callers that must not
 * allocate device memory: code that draws all of its device memory from a host
 * application's own pool or budget, latency-critical code that cannot afford the implicit
 * device-wide synchronisation of cudaMalloc / cudaFree, and plugins that are handed device
 * buffers but not the right to allocate.  Everything else in this library allocates.
 *
 * Static PageRank (the same computation as pr_static: ranks iterated from 1/n until the
 * L-inf change is <= params->tol or params->max_iter iterations ran) of a graph given as
 * an in-edge CSR in device memory: in_off[0..n] (non-decreasing from 0 to m) and
 * in_col[0..m) = the sources u of the edges (u, v) of row v, in the layout
 * pr_get_csr(g, 1, ...) exports.  Every vertex needs an out-edge (a self-loop on every
 * vertex gives one).  The n ranks are written to `ranks` (device memory); the work runs on
 * cuda_stream and the call is synchronous: it returns when that work has finished.
 * params may be NULL (defaults); it must ask for PR_F64 and PR_DEADEND_SELFLOOP.  stats
 * may be NULL; its timing fields stay 0.  Arithmetic is plain FP64, so the ranks agree
 * with pr_static's within the usual L-inf tolerance, not bit for bit.
 *
 * No device memory is allocated.  Working memory is one fixed array of
 * PR_NOALLOC_SCRATCH_BYTES inside this library, held on every device that loads the
 * library until the process exits; hence n <= PR_NOALLOC_MAX_VERTICES, and larger n is
 * rejected with PR_ERR_CAPACITY before any device work.  The first call on a device looks
 * up that array's device address (with that device current), so make the first call on
 * each device before any stream capture begins.  All calls on a device share the array:
 * calls whose work overlaps on the GPU (several host threads, or several streams) race and
 * must be serialised by the caller.  A call clears what it needs cleared at its start.
 * Errors: PR_ERR_INVALID_ARG (NULL or host pointers, pointers on another device than the
 * current one, bad params, malformed offsets, a vertex with no out-edge),
 * PR_ERR_VERTEX_RANGE (a column id >= n), PR_ERR_CUDA; ranks are written only after the
 * CSR has passed these checks. */
#define PR_NOALLOC_MAX_VERTICES (1u << 18)
#define PR_NOALLOC_SCRATCH_BYTES (256u + 20u * PR_NOALLOC_MAX_VERTICES)
pr_status pr_static_noalloc(uint32_t n, int64_t m, const uint64_t *in_off, const uint32_t *in_col,
                            const pr_params *params, void *cuda_stream, double *ranks, pr_stats *stats);

/* ---------------------------------------------------------------- serving form ----
 * A request loop over several resident graphs.  Each attached graph gets a FIFO and one
 * worker, so it has a single writer and its requests run in submission order; requests of
 * different graphs run concurrently on their graphs' streams (create each graph with its
 * own stream for overlap).  A request is admitted when one of `slots` device slots is free
 * and free device memory (cudaMemGetInfo) covers hbm_reserve_bytes plus the request's
 * estimate; an idle device always admits one request.  Attaching a graph sizes its
 * persistent launch to 1/slots of the resident blocks so concurrent launches fit together.
 * An update = one pr_apply_batches over the coalesced requests in submission order + one
 * pr_dynamic_frontier;
 * results carry host-clock times in ms since the server was created.  While attached, a
 * graph must not be used directly. */
typedef struct pr_server pr_server;

typedef struct {
    int32_t slots;               /* concurrent updates on the device (1..64) */
    int32_t max_coalesce;        /* queued requests of one graph served by one update (>= 1):
                                    their batches are applied in order by one
                                    pr_apply_batches, then one Dynamic Frontier call covers
                                    the net change */
    uint64_t hbm_reserve_bytes;  /* device memory to keep free */
} pr_server_config;

typedef struct {
    uint64_t ticket;
    int32_t graph;               /* index from pr_server_add_graph */
    int32_t status;              /* pr_status of the request */
    double t_submit_ms, t_start_ms, t_done_ms;
    int32_t coalesced;           /* requests served by the same update (1 = alone) */
    int32_t reserved;
    pr_stats stats;              /* of the pr_dynamic_frontier that served it */
} pr_request_result;

typedef struct {
    int64_t submitted, completed, waited_for_memory;
    double elapsed_ms;
} pr_server_info;

void pr_server_config_default(pr_server_config *cfg); /* 2 slots, coalesce up to 256, 1 GiB reserve */
pr_status pr_server_create(const pr_server_config *cfg, pr_server **out);
/* Attaches g (caller keeps ownership; destroy the server before the graph). */
pr_status pr_server_add_graph(pr_server *s, pr_graph *g, int32_t *index);
/* Queues one batch for graph `graph` (host arrays, copied); returns at once with a ticket. */
pr_status pr_server_submit(pr_server *s, int32_t graph, int64_t n_del, const uint32_t *del_src,
                           const uint32_t *del_dst, int64_t n_ins, const uint32_t *ins_src, const uint32_t *ins_dst,
                           uint64_t *ticket);
/* Blocks until the request has finished and copies its result. */
pr_status pr_server_wait(pr_server *s, uint64_t ticket, pr_request_result *out);
/* Blocks until every submitted request has finished; info may be NULL. */
pr_status pr_server_drain(pr_server *s, pr_server_info *info);
/* Finishes queued requests, joins the workers and frees the server (not the graphs). */
pr_status pr_server_destroy(pr_server *s);

/* Message of the last failed call on g (or of the last failed pr_graph_create if g is NULL). */
const char *pr_last_error(const pr_graph *g);

/* Short name of a status code. */
const char *pr_status_string(pr_status s);

#ifdef __cplusplus
}
#endif

#endif /* PRDF_H */

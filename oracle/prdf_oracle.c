/*
 * prdf_oracle.c - plain, sequential FP64 oracle for Dynamic Frontier PageRank.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load this library.  It shares no code with the CUDA library: no
 * headers, no helpers, no tables.  It is deliberately slow and literal so that each
 * function can be checked against the paper by eye.
 *
 * Paper: S. Sahu, "An Incrementally Expanding Approach for Updating PageRank on
 * Dynamic Graphs" (arXiv 2401.03256).
 *
 *   or_graph_build      Section 3.1 (self-loops on every vertex against dead ends),
 *                       Section 5.1.4 (self-loops re-added with every batch).
 *   or_apply_batch      Section 3.2: E^t = (E^{t-1} \ D) U I, and the effective
 *                       Delta^- = E^{t-1} \ E^t, Delta^+ = E^t \ E^{t-1}.
 *   or_static           Section 3.1, Eq. 1: power iteration from 1/n, L-inf test.
 *   or_naive            Section 3.3.1: the same sweep started from previous ranks.
 *   or_df_sync          Algorithm 1 with the synchronous (two-vector, Jacobi) reading
 *                       of Section 4.2: marks made in iteration i take effect in i+1.
 *   or_dt_sync          Dynamic Traversal (Section 3.3.2): vertices reachable from the
 *                       changed edges' sources in G^{t-1} or G^t, iterated synchronously.
 *   or_df_async         Algorithm 1 with the asynchronous (one-vector) reading of
 *                       Section 4.2: vertices swept in ascending id, in place, marks
 *                       take effect at once.  The paper's CPU choice.
 *   or_dense_solve      Direct solve of (I - alpha P^T) r = (1 - alpha)/n with dead-end
 *                       teleport, Gaussian elimination in long double.
 *
 * Dead ends (Section 3.1): with self-loops (mode 0) no vertex has out-degree 0.  In
 * teleport mode (mode 1) no self-loops are added and a dead end u spreads its rank over
 * all n vertices: R[v] gets alpha * D / n with D = sum of R over dead ends.
 *
 * Threads: the vertex loops of the synchronous sweeps carry OpenMP annotations
 * (schedule(dynamic, 2048), the paper's CPU schedule, Section 5.1.2).  The parity oracle
 * is built without -fopenmp, so they are ignored and every loop runs in order.  A second
 * build with -fopenmp times the same code on all host cores; it gives the same results
 * bit for bit, because each vertex's sum is still taken by one thread in in-edge order,
 * the L-inf maximum is exact, and marking only sets flags to 1.  The asynchronous
 * reading (or_df_async) is never parallel: its result depends on the sweep order.
 *
 * Parity notes for dynamic frontier with teleport (the paper avoids this mode): D is
 * recomputed at the start of every iteration from that iteration's input ranks; if
 * alpha * |D - D_prev| / n exceeds the frontier tolerance, every vertex is marked
 * affected from that iteration on (D_prev of iteration 0 is the previous graph's dead-end
 * mass under the previous ranks).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    uint32_t n;
    uint64_t m;          /* edges, including the added self-loops */
    int self_loops;      /* 1 if a self-loop was added to every vertex */
    uint64_t *out_off;   /* n + 1 */
    uint32_t *out_col;   /* m; each row ascending */
    uint64_t *in_off;    /* n + 1 */
    uint32_t *in_col;    /* m; each row ascending */
} or_graph;

typedef struct {
    double alpha;          /* damping factor, 0.85 (Section 5.1.2) */
    double tol;            /* iteration tolerance tau on the L-inf norm, 1e-10 */
    double frontier_tol;   /* frontier tolerance tau_f = tau / 1e5 (Section 4.3) */
    int32_t max_iter;      /* MAX_ITERATIONS, 500 */
    int32_t dead_end;      /* 0: self-loops, 1: global teleport */
} or_params;

typedef struct {
    int32_t iterations;
    int32_t converged;
    int64_t affected_final;
    int64_t vertices_processed;
    int64_t edges_processed;
    double last_delta;
} or_stats;

/* Threads of the vertex loops: 1 in the sequential build; in the -fopenmp build k > 0
 * sets the count.  Returns the count in effect. */
int or_threads(int k)
{
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
    return omp_get_max_threads();
#else
    (void)k;
    return 1;
#endif
}

/* ------------------------------------------------------------------ graph ---- */

static int cmp_u64(const void *x, const void *y)
{
    uint64_t a = *(const uint64_t *)x, b = *(const uint64_t *)y;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* Sorted, unique keys (u << 32 | v) of the given pairs with u != v. */
static uint64_t *pair_set(uint64_t k, const uint32_t *src, const uint32_t *dst, uint64_t *count)
{
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (k ? k : 1));
    uint64_t w = 0;
    for (uint64_t i = 0; i < k; i++)
        if (src[i] != dst[i]) keys[w++] = ((uint64_t)src[i] << 32) | dst[i];
    qsort(keys, w, sizeof(uint64_t), cmp_u64);
    uint64_t u = 0;
    for (uint64_t i = 0; i < w; i++)
        if (u == 0 || keys[u - 1] != keys[i]) keys[u++] = keys[i];
    *count = u;
    return keys;
}

static int has_key(const uint64_t *a, uint64_t n, uint64_t x)
{
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo < n && a[lo] == x;
}

/* Union of two ascending key arrays without repeats (a and b each have none). */
static uint64_t merge_sets(const uint64_t *a, uint64_t na, const uint64_t *b, uint64_t nb, uint64_t *out)
{
    uint64_t i = 0, j = 0, w = 0;
    while (i < na || j < nb) {
        if (j >= nb || (i < na && a[i] < b[j])) out[w++] = a[i++];
        else if (i >= na || b[j] < a[i]) out[w++] = b[j++];
        else { out[w++] = a[i++]; j++; }
    }
    return w;
}

/* Build both adjacencies from a sorted unique key set E (no self pairs); adds the
 * self-loop (v, v) of every vertex if self_loops is set.  Takes ownership of nothing. */
static or_graph *graph_from_set(uint32_t n, const uint64_t *E, uint64_t e, int self_loops)
{
    or_graph *g = (or_graph *)calloc(1, sizeof(or_graph));
    g->n = n;
    g->self_loops = self_loops;
    g->m = e + (self_loops ? n : 0);
    uint64_t *all = (uint64_t *)malloc(sizeof(uint64_t) * (g->m ? g->m : 1));
    if (self_loops) {
        uint64_t *loops = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
        for (uint32_t v = 0; v < n; v++) loops[v] = ((uint64_t)v << 32) | v;
        merge_sets(E, e, loops, n, all);
        free(loops);
    } else {
        memcpy(all, E, sizeof(uint64_t) * e);
    }

    /* out-adjacency: rows by source, each row ascending by target */
    g->out_off = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    g->out_col = (uint32_t *)malloc(sizeof(uint32_t) * (g->m ? g->m : 1));
    for (uint64_t i = 0; i < g->m; i++) g->out_off[(all[i] >> 32) + 1]++;
    for (uint32_t v = 0; v < n; v++) g->out_off[v + 1] += g->out_off[v];
    for (uint64_t i = 0; i < g->m; i++) g->out_col[i] = (uint32_t)all[i];

    /* in-adjacency: rows by target; walking the (source, target)-sorted list in order
     * and appending keeps each row ascending by source */
    g->in_off = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    g->in_col = (uint32_t *)malloc(sizeof(uint32_t) * (g->m ? g->m : 1));
    for (uint64_t i = 0; i < g->m; i++) g->in_off[(uint32_t)all[i] + 1]++;
    for (uint32_t v = 0; v < n; v++) g->in_off[v + 1] += g->in_off[v];
    uint64_t *fill = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    memcpy(fill, g->in_off, sizeof(uint64_t) * ((size_t)n + 1));
    for (uint64_t i = 0; i < g->m; i++) {
        uint32_t v = (uint32_t)all[i];
        g->in_col[fill[v]++] = (uint32_t)(all[i] >> 32);
    }
    free(fill);
    free(all);
    return g;
}

/* Edge set of g without the added self-loops, as sorted keys. */
static uint64_t *graph_edge_set(const or_graph *g, uint64_t *count)
{
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (g->m ? g->m : 1));
    uint64_t w = 0;
    for (uint32_t u = 0; u < g->n; u++)
        for (uint64_t j = g->out_off[u]; j < g->out_off[u + 1]; j++)
            if (g->out_col[j] != u) keys[w++] = ((uint64_t)u << 32) | g->out_col[j];
    *count = w;
    return keys;
}

/* Returns NULL if an id is out of range. */
or_graph *or_graph_build(uint32_t n, uint64_t k, const uint32_t *src, const uint32_t *dst,
                         int self_loops)
{
    for (uint64_t i = 0; i < k; i++)
        if (src[i] >= n || dst[i] >= n) return NULL;
    uint64_t e;
    uint64_t *E = pair_set(k, src, dst, &e);
    or_graph *g = graph_from_set(n, E, e, self_loops);
    free(E);
    return g;
}

void or_graph_free(or_graph *g)
{
    if (!g) return;
    free(g->out_off); free(g->out_col); free(g->in_off); free(g->in_col);
    free(g);
}

uint32_t or_graph_n(const or_graph *g) { return g->n; }
uint64_t or_graph_m(const or_graph *g) { return g->m; }

/* dir 0: out-adjacency, 1: in-adjacency.  off has n + 1 entries, col has m. */
void or_graph_export(const or_graph *g, int dir, uint64_t *off, uint32_t *col)
{
    const uint64_t *o = dir ? g->in_off : g->out_off;
    const uint32_t *c = dir ? g->in_col : g->out_col;
    memcpy(off, o, sizeof(uint64_t) * ((size_t)g->n + 1));
    memcpy(col, c, sizeof(uint32_t) * g->m);
}

/*
 * Section 3.2: E^t = (E^{t-1} \ D) U I with D, I the requested deletions and
 * insertions (pairs u == v ignored: self-loops are fixed).  Writes the effective
 * Delta^- = E^{t-1} \ E^t and Delta^+ = E^t \ E^{t-1} (sorted by (u, v)) into the
 * caller's arrays (capacities nd and ni) and returns the new graph; the old graph is
 * left unchanged.  Returns NULL if an id is out of range.
 */
or_graph *or_apply_batch(const or_graph *g, uint64_t nd, const uint32_t *ds, const uint32_t *dd,
                         uint64_t ni, const uint32_t *is, const uint32_t *id,
                         uint64_t *n_eff_del, uint32_t *eds, uint32_t *edd,
                         uint64_t *n_eff_ins, uint32_t *eis, uint32_t *eid)
{
    for (uint64_t i = 0; i < nd; i++) if (ds[i] >= g->n || dd[i] >= g->n) return NULL;
    for (uint64_t i = 0; i < ni; i++) if (is[i] >= g->n || id[i] >= g->n) return NULL;
    uint64_t e_old, c_del, c_ins;
    uint64_t *E = graph_edge_set(g, &e_old);
    uint64_t *D = pair_set(nd, ds, dd, &c_del);
    uint64_t *I = pair_set(ni, is, id, &c_ins);

    /* E minus D, then union with I (all ascending) */
    uint64_t *Ekeep = (uint64_t *)malloc(sizeof(uint64_t) * (e_old + 1));
    uint64_t w = 0;
    for (uint64_t i = 0; i < e_old; i++)
        if (!has_key(D, c_del, E[i])) Ekeep[w++] = E[i];
    uint64_t *Enew = (uint64_t *)malloc(sizeof(uint64_t) * (w + c_ins + 1));
    uint64_t e_new = merge_sets(Ekeep, w, I, c_ins, Enew);
    free(Ekeep);

    /* Delta^- = E^{t-1} \ E^t and Delta^+ = E^t \ E^{t-1}, by one walk over both sets */
    uint64_t a = 0, b = 0, i = 0, j = 0;
    while (i < e_old || j < e_new) {
        if (j >= e_new || (i < e_old && E[i] < Enew[j])) {
            eds[a] = (uint32_t)(E[i] >> 32); edd[a] = (uint32_t)E[i]; a++; i++;
        } else if (i >= e_old || Enew[j] < E[i]) {
            eis[b] = (uint32_t)(Enew[j] >> 32); eid[b] = (uint32_t)Enew[j]; b++; j++;
        } else {
            i++; j++;
        }
    }
    *n_eff_del = a;
    *n_eff_ins = b;

    or_graph *h = graph_from_set(g->n, Enew, e_new, g->self_loops);
    free(E); free(D); free(I); free(Enew);
    return h;
}

/* --------------------------------------------------------------- pagerank ---- */

static uint64_t out_degree(const or_graph *g, uint32_t u) { return g->out_off[u + 1] - g->out_off[u]; }

/* D = sum of R over the dead ends of g (zero with self-loops). */
static double dead_end_mass(const or_graph *g, const double *R)
{
    double D = 0.0;
    for (uint32_t u = 0; u < g->n; u++)
        if (out_degree(g, u) == 0) D += R[u];
    return D;
}

/* Eq. 1 for one vertex: r = (1 - alpha)/n + sum over u in in(v) of alpha R[u] / |out(u)|,
 * accumulated in the order of Algorithm 1; teleport mode adds alpha D / n. */
static double rank_of(const or_graph *g, const or_params *p, const double *R, uint32_t v, double D)
{
    double r = (1.0 - p->alpha) / (double)g->n;
    for (uint64_t j = g->in_off[v]; j < g->in_off[v + 1]; j++) {
        uint32_t u = g->in_col[j];
        r = r + p->alpha * R[u] / (double)out_degree(g, u);
    }
    if (p->dead_end == 1) r = r + p->alpha * D / (double)g->n;
    return r;
}

/* Power iteration over all vertices, Jacobi (two vectors), until the L-inf change is
 * at most tau or max_iter sweeps were made. */
static void sweep_until_converged(const or_graph *g, const or_params *p, double *R, or_stats *st)
{
    uint32_t n = g->n;
    double *Rn = (double *)malloc(sizeof(double) * (n ? n : 1));
    st->iterations = 0;
    st->converged = 0;
    st->last_delta = 0.0;
    st->vertices_processed = 0;
    st->edges_processed = 0;
    for (int32_t i = 0; i < p->max_iter; i++) {
        double D = p->dead_end == 1 ? dead_end_mass(g, R) : 0.0;
        double dR = 0.0;
        int64_t edges = 0;
        #pragma omp parallel for schedule(dynamic, 2048) reduction(max : dR) reduction(+ : edges)
        for (uint32_t v = 0; v < n; v++) {
            double r = rank_of(g, p, R, v, D);
            double d = fabs(r - R[v]);
            if (d > dR) dR = d;
            Rn[v] = r;
            edges += (int64_t)(g->in_off[v + 1] - g->in_off[v]);
        }
        st->edges_processed += edges;
        st->vertices_processed += n;
        memcpy(R, Rn, sizeof(double) * n);
        st->iterations = i + 1;
        st->last_delta = dR;
        if (dR <= p->tol) { st->converged = 1; break; }
    }
    st->affected_final = n;
    free(Rn);
}

/* Static PageRank (Section 3.1): R starts at 1/n. */
int or_static(const or_graph *g, const or_params *p, double *R, or_stats *st)
{
    for (uint32_t v = 0; v < g->n; v++) R[v] = 1.0 / (double)g->n;
    sweep_until_converged(g, p, R, st);
    return 0;
}

/* Naive-dynamic PageRank (Section 3.3.1): R holds the previous ranks on entry. */
int or_naive(const or_graph *g, const or_params *p, double *R, or_stats *st)
{
    sweep_until_converged(g, p, R, st);
    return 0;
}

/* Algorithm 1, initial marking: for every (u, v) in Delta^- U Delta^+ mark each
 * v' in G^{t-1}.out(u) and in G^t.out(u). */
static void mark_initial(const or_graph *gold, const or_graph *gnew,
                         uint64_t nd, const uint32_t *ds,
                         uint64_t ni, const uint32_t *is, uint8_t *aff)
{
    for (uint64_t k = 0; k < nd + ni; k++) {
        uint32_t u = k < nd ? ds[k] : is[k - nd];
        for (uint64_t j = gold->out_off[u]; j < gold->out_off[u + 1]; j++) aff[gold->out_col[j]] = 1;
        for (uint64_t j = gnew->out_off[u]; j < gnew->out_off[u + 1]; j++) aff[gnew->out_col[j]] = 1;
    }
}

static int64_t count_marked(const uint8_t *aff, uint32_t n)
{
    int64_t c = 0;
    for (uint32_t v = 0; v < n; v++) c += aff[v] ? 1 : 0;
    return c;
}

/*
 * Algorithm 1, synchronous reading.  gold = G^{t-1}, gnew = G^t; (ds, dd) and (is, id)
 * are the effective Delta^- and Delta^+; R holds R^{t-1} on entry and R on exit.
 * aff (n bytes, may be NULL) receives the final affected flags.
 *
 * Each iteration: every affected v gets r from the iteration's input ranks; the
 * L-inf change is the max of |r - R[v]|; if |r - R[v]| > tau_f the out-neighbours of
 * v in G^t are marked for the next iteration; the new ranks replace the old ones
 * together; stop when the change is at most tau.
 */
int or_df_sync(const or_graph *gold, const or_graph *gnew, const or_params *p,
               uint64_t nd, const uint32_t *ds, const uint32_t *dd,
               uint64_t ni, const uint32_t *is, const uint32_t *id,
               double *R, uint8_t *aff_out, or_stats *st)
{
    (void)dd; (void)id;
    uint32_t n = gnew->n;
    uint8_t *aff = (uint8_t *)calloc(n ? n : 1, 1);
    uint8_t *next = (uint8_t *)calloc(n ? n : 1, 1);
    double *Rn = (double *)malloc(sizeof(double) * (n ? n : 1));
    memset(st, 0, sizeof(*st));

    mark_initial(gold, gnew, nd, ds, ni, is, aff);
    double D_prev = p->dead_end == 1 ? dead_end_mass(gold, R) : 0.0;

    for (int32_t i = 0; i < p->max_iter; i++) {
        double D = 0.0;
        if (p->dead_end == 1) {
            D = dead_end_mass(gnew, R);
            if (p->alpha * fabs(D - D_prev) / (double)n > p->frontier_tol)
                for (uint32_t v = 0; v < n; v++) aff[v] = 1;
            D_prev = D;
        }
        memcpy(next, aff, n);
        memcpy(Rn, R, sizeof(double) * n);
        double dR = 0.0;
        int64_t verts = 0, edges = 0;
        #pragma omp parallel for schedule(dynamic, 2048) reduction(max : dR) reduction(+ : verts, edges)
        for (uint32_t v = 0; v < n; v++) {
            if (!aff[v]) continue;
            double r = rank_of(gnew, p, R, v, D);
            double d = fabs(r - R[v]);
            Rn[v] = r;
            if (d > dR) dR = d;
            if (d > p->frontier_tol)
                for (uint64_t j = gnew->out_off[v]; j < gnew->out_off[v + 1]; j++)
                    __atomic_store_n(&next[gnew->out_col[j]], (uint8_t)1, __ATOMIC_RELAXED);
            verts++;
            edges += (int64_t)(gnew->in_off[v + 1] - gnew->in_off[v]);
        }
        st->vertices_processed += verts;
        st->edges_processed += edges;
        memcpy(R, Rn, sizeof(double) * n);
        memcpy(aff, next, n);
        st->iterations = i + 1;
        st->last_delta = dR;
        if (dR <= p->tol) { st->converged = 1; break; }
    }
    st->affected_final = count_marked(aff, n);
    if (aff_out) memcpy(aff_out, aff, n);
    free(aff); free(next); free(Rn);
    return 0;
}

/*
 * Dynamic Traversal (Section 3.3.2, the comparator of Section 5): for every (u, v) in
 * Delta^- U Delta^+, every vertex reachable from u in G^{t-1} or in G^t is affected
 * (breadth-first search in each graph separately; a vertex reaches itself).  The affected
 * vertices are then iterated as in or_df_sync, but nothing further is ever marked.  In
 * teleport mode a changed dead-end mass moves every rank, so every vertex is affected.
 */
static void reach(const or_graph *g, uint32_t u, uint8_t *seen, uint32_t *queue)
{
    if (seen[u]) return;
    uint64_t head = 0, tail = 0;
    seen[u] = 1;
    queue[tail++] = u;
    while (head < tail) {
        uint32_t x = queue[head++];
        for (uint64_t j = g->out_off[x]; j < g->out_off[x + 1]; j++) {
            uint32_t w = g->out_col[j];
            if (!seen[w]) {
                seen[w] = 1;
                queue[tail++] = w;
            }
        }
    }
}

int or_dt_sync(const or_graph *gold, const or_graph *gnew, const or_params *p,
               uint64_t nd, const uint32_t *ds, const uint32_t *dd,
               uint64_t ni, const uint32_t *is, const uint32_t *id,
               double *R, uint8_t *aff_out, or_stats *st)
{
    (void)dd; (void)id;
    uint32_t n = gnew->n;
    uint8_t *seen_old = (uint8_t *)calloc(n ? n : 1, 1);
    uint8_t *seen_new = (uint8_t *)calloc(n ? n : 1, 1);
    uint8_t *aff = (uint8_t *)calloc(n ? n : 1, 1);
    uint32_t *queue = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    double *Rn = (double *)malloc(sizeof(double) * (n ? n : 1));
    memset(st, 0, sizeof(*st));
    for (uint64_t k = 0; k < nd + ni; k++) {
        uint32_t u = k < nd ? ds[k] : is[k - nd];
        reach(gold, u, seen_old, queue);
        reach(gnew, u, seen_new, queue);
    }
    for (uint32_t v = 0; v < n; v++) aff[v] = (uint8_t)(seen_old[v] | seen_new[v]);
    if (p->dead_end == 1 && nd + ni > 0)
        for (uint32_t v = 0; v < n; v++) aff[v] = 1;
    for (int32_t i = 0; i < p->max_iter; i++) {
        double D = p->dead_end == 1 ? dead_end_mass(gnew, R) : 0.0;
        memcpy(Rn, R, sizeof(double) * n);
        double dR = 0.0;
        int64_t verts = 0, edges = 0;
        #pragma omp parallel for schedule(dynamic, 2048) reduction(max : dR) reduction(+ : verts, edges)
        for (uint32_t v = 0; v < n; v++) {
            if (!aff[v]) continue;
            double r = rank_of(gnew, p, R, v, D);
            double d = fabs(r - R[v]);
            Rn[v] = r;
            if (d > dR) dR = d;
            verts++;
            edges += (int64_t)(gnew->in_off[v + 1] - gnew->in_off[v]);
        }
        st->vertices_processed += verts;
        st->edges_processed += edges;
        memcpy(R, Rn, sizeof(double) * n);
        st->iterations = i + 1;
        st->last_delta = dR;
        if (dR <= p->tol) { st->converged = 1; break; }
    }
    st->affected_final = count_marked(aff, n);
    if (aff_out) memcpy(aff_out, aff, n);
    free(seen_old); free(seen_new); free(aff); free(queue); free(Rn);
    return 0;
}

/*
 * Algorithm 1, asynchronous reading (Section 4.2): one rank vector updated in place,
 * affected vertices swept in ascending id, marks visible immediately (a vertex marked
 * ahead of the sweep is processed in the same iteration).
 */
int or_df_async(const or_graph *gold, const or_graph *gnew, const or_params *p,
                uint64_t nd, const uint32_t *ds, const uint32_t *dd,
                uint64_t ni, const uint32_t *is, const uint32_t *id,
                double *R, uint8_t *aff_out, or_stats *st)
{
    (void)dd; (void)id;
    uint32_t n = gnew->n;
    uint8_t *aff = (uint8_t *)calloc(n ? n : 1, 1);
    memset(st, 0, sizeof(*st));
    mark_initial(gold, gnew, nd, ds, ni, is, aff);
    double D_prev = p->dead_end == 1 ? dead_end_mass(gold, R) : 0.0;

    for (int32_t i = 0; i < p->max_iter; i++) {
        double D = 0.0;
        if (p->dead_end == 1) {
            D = dead_end_mass(gnew, R);
            if (p->alpha * fabs(D - D_prev) / (double)n > p->frontier_tol)
                for (uint32_t v = 0; v < n; v++) aff[v] = 1;
            D_prev = D;
        }
        double dR = 0.0;
        for (uint32_t v = 0; v < n; v++) {
            if (!aff[v]) continue;
            double r = rank_of(gnew, p, R, v, D);
            double d = fabs(r - R[v]);
            R[v] = r;
            if (d > dR) dR = d;
            if (d > p->frontier_tol)
                for (uint64_t j = gnew->out_off[v]; j < gnew->out_off[v + 1]; j++) aff[gnew->out_col[j]] = 1;
            st->vertices_processed++;
            st->edges_processed += (int64_t)(gnew->in_off[v + 1] - gnew->in_off[v]);
        }
        st->iterations = i + 1;
        st->last_delta = dR;
        if (dR <= p->tol) { st->converged = 1; break; }
    }
    st->affected_final = count_marked(aff, n);
    if (aff_out) memcpy(aff_out, aff, n);
    free(aff);
    return 0;
}

/* -------------------------------------------------------------- dense solve ---- */

/*
 * Solves (I - alpha P^T) r = (1 - alpha)/n * 1 for a small graph given as pairs (pairs
 * u == v and duplicates ignored; self-loops added if self_loops).  P[u][v] = 1/|out(u)|
 * for an edge u -> v; a dead end u has P[u][v] = 1/n for every v.  Gaussian
 * elimination with partial pivoting in long double.  Returns 0, or -1 on a bad id,
 * n > 4096, or a singular pivot.
 */
int or_dense_solve(uint32_t n, uint64_t k, const uint32_t *src, const uint32_t *dst,
                   int self_loops, double alpha, double *r_out)
{
    if (n == 0 || n > 4096) return -1;
    for (uint64_t i = 0; i < k; i++) if (src[i] >= n || dst[i] >= n) return -1;
    size_t N = n;
    uint8_t *adj = (uint8_t *)calloc(N * N, 1);       /* adj[u*N + v] = edge u -> v */
    for (uint64_t i = 0; i < k; i++) if (src[i] != dst[i]) adj[(size_t)src[i] * N + dst[i]] = 1;
    if (self_loops) for (size_t v = 0; v < N; v++) adj[v * N + v] = 1;
    long double *A = (long double *)calloc(N * (N + 1), sizeof(long double));  /* [N][N+1] */
    for (size_t v = 0; v < N; v++) A[v * (N + 1) + v] = 1.0L;
    for (size_t u = 0; u < N; u++) {
        size_t d = 0;
        for (size_t v = 0; v < N; v++) d += adj[u * N + v];
        for (size_t v = 0; v < N; v++) {
            long double puv = d ? (adj[u * N + v] ? 1.0L / (long double)d : 0.0L) : 1.0L / (long double)N;
            A[v * (N + 1) + u] -= (long double)alpha * puv;   /* row v, column u: (P^T)[v][u] */
        }
    }
    for (size_t v = 0; v < N; v++) A[v * (N + 1) + N] = (1.0L - (long double)alpha) / (long double)N;
    int rc = 0;
    for (size_t c = 0; c < N && rc == 0; c++) {
        size_t piv = c;
        for (size_t r = c + 1; r < N; r++)
            if (fabsl(A[r * (N + 1) + c]) > fabsl(A[piv * (N + 1) + c])) piv = r;
        if (fabsl(A[piv * (N + 1) + c]) < 1e-30L) { rc = -1; break; }
        if (piv != c)
            for (size_t j = 0; j <= N; j++) {
                long double t = A[c * (N + 1) + j];
                A[c * (N + 1) + j] = A[piv * (N + 1) + j];
                A[piv * (N + 1) + j] = t;
            }
        for (size_t r = c + 1; r < N; r++) {
            long double f = A[r * (N + 1) + c] / A[c * (N + 1) + c];
            if (f == 0.0L) continue;
            for (size_t j = c; j <= N; j++) A[r * (N + 1) + j] -= f * A[c * (N + 1) + j];
        }
    }
    if (rc == 0) {
        long double *x = (long double *)calloc(N, sizeof(long double));
        for (size_t c = N; c-- > 0;) {
            long double s = A[c * (N + 1) + N];
            for (size_t j = c + 1; j < N; j++) s -= A[c * (N + 1) + j] * x[j];
            x[c] = s / A[c * (N + 1) + c];
        }
        for (size_t v = 0; v < N; v++) r_out[v] = (double)x[v];
        free(x);
    }
    free(adj);
    free(A);
    return rc;
}

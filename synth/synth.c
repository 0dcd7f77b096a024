/*
 * synth.c - seeded synthetic inputs for Dynamic Frontier PageRank.
 *
 * This module produces INPUTS only: directed graphs and batch updates with the
 * shapes of the paper's workloads (R-MAT / Kronecker power-law graphs, a road-like
 * grid, uniformly random 80/20 insertion/deletion batches, Section 5.1.4).  It holds
 * none of the method's arithmetic: no ranks, no CSR, no marking.  Both the oracle and
 * the CUDA library consume what it writes, and neither of them is linked into it.
 *
 * Random numbers: splitmix64 (Steele, Lea, Flood 2014) seeds xoshiro256** (Blackman,
 * Vigna 2018).  A 32-bit uniform is the top half of one xoshiro output, a double the
 * top 53 bits.  Work is cut into fixed chunks of samples, each with its own stream, so
 * the output does not depend on the number of threads.
 *
 * Edge keys are (u << 32) | v, so sorting keys sorts edges by (source, target).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GOLDEN 0x9E3779B97F4A7C15ULL

static uint64_t splitmix64_next(uint64_t *state)
{
    uint64_t z = (*state += GOLDEN);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } xrng;

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t xr_next(xrng *r)
{
    uint64_t *s = r->s;
    uint64_t out = rotl64(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return out;
}

static void xr_seed(xrng *r, uint64_t seed)
{
    uint64_t st = seed;
    for (int i = 0; i < 4; i++) r->s[i] = splitmix64_next(&st);
}

/* Unbiased integer in [0, bound) by rejection on the top bits (bound >= 1). */
static inline uint64_t xr_below(xrng *r, uint64_t bound)
{
    if (bound <= 1) return 0;
    uint64_t mask = bound - 1;
    mask |= mask >> 1; mask |= mask >> 2; mask |= mask >> 4;
    mask |= mask >> 8; mask |= mask >> 16; mask |= mask >> 32;
    for (;;) {
        uint64_t x = xr_next(r) & mask;
        if (x < bound) return x;
    }
}

/* Seed of stream `idx` derived from a base seed (one splitmix step over a mixed word). */
static uint64_t sub_seed(uint64_t seed, uint64_t idx)
{
    uint64_t st = seed ^ ((idx + 1) * GOLDEN);
    return splitmix64_next(&st);
}

/* ---------------------------------------------------------------- sorting ---- */

/* LSD radix sort of 64-bit keys on 16-bit digits; digits that are equal in every key
 * are skipped.  tmp must hold n keys.  Result ends in keys. */
static void radix_sort_u64(uint64_t *keys, uint64_t *tmp, uint64_t n)
{
    if (n < 2) return;
    uint64_t *cnt = (uint64_t *)malloc(sizeof(uint64_t) * 65536);
    uint64_t *src = keys, *dst = tmp;
    for (int shift = 0; shift < 64; shift += 16) {
        memset(cnt, 0, sizeof(uint64_t) * 65536);
        for (uint64_t i = 0; i < n; i++) cnt[(src[i] >> shift) & 0xFFFF]++;
        int single = 0;
        for (int d = 0; d < 65536; d++) if (cnt[d] == n) { single = 1; break; }
        if (single) continue;
        uint64_t run = 0;
        for (int d = 0; d < 65536; d++) { uint64_t c = cnt[d]; cnt[d] = run; run += c; }
        for (uint64_t i = 0; i < n; i++) dst[cnt[(src[i] >> shift) & 0xFFFF]++] = src[i];
        uint64_t *t = src; src = dst; dst = t;
    }
    if (src != keys) memcpy(keys, src, sizeof(uint64_t) * n);
    free(cnt);
}

/* Sort, drop duplicates and self-pairs (u == v); returns the new count. */
static uint64_t sort_unique_no_self(uint64_t *keys, uint64_t n)
{
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
    radix_sort_u64(keys, tmp, n);
    free(tmp);
    uint64_t w = 0;
    for (uint64_t i = 0; i < n; i++) {
        uint64_t k = keys[i];
        if ((uint32_t)(k >> 32) == (uint32_t)k) continue;
        if (w > 0 && keys[w - 1] == k) continue;
        keys[w++] = k;
    }
    return w;
}

static int64_t lower_bound_u64(const uint64_t *a, int64_t n, uint64_t x)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

static int contains_u64(const uint64_t *a, int64_t n, uint64_t x)
{
    int64_t p = lower_bound_u64(a, n, x);
    return p < n && a[p] == x;
}

/* ------------------------------------------------------------- generators ---- */

#define RMAT_CHUNK (1ULL << 16)

/*
 * R-MAT / Kronecker sampler (Chakrabarti, Zhan, Faloutsos 2004).  Draws ef * 2^scale
 * directed pairs; at each of `scale` bit levels one 32-bit uniform picks the quadrant
 * with probabilities (a, b, c, 1-a-b-c).  If `permute` is set, vertex ids are relabelled
 * by one seeded uniform permutation so hubs do not sit at low ids.  Self-pairs and
 * duplicates are removed.  Output: sorted unique keys, count in *m_out; caller frees
 * with synth_free.  Returns NULL on allocation failure.
 */
uint64_t *synth_rmat(int scale, double ef, double a, double b, double c, uint64_t seed,
                     int permute, uint64_t *m_out)
{
    uint64_t n = 1ULL << scale;
    uint64_t samples = (uint64_t)llround(ef * (double)n);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (samples ? samples : 1));
    if (!keys) return NULL;
    uint32_t ta = (uint32_t)fmin(4294967295.0, floor(a * 4294967296.0));
    uint32_t tb = (uint32_t)fmin(4294967295.0, floor((a + b) * 4294967296.0));
    uint32_t tc = (uint32_t)fmin(4294967295.0, floor((a + b + c) * 4294967296.0));
    uint64_t nchunks = (samples + RMAT_CHUNK - 1) / RMAT_CHUNK;

    uint32_t *perm = NULL;
    if (permute) {
        perm = (uint32_t *)malloc(sizeof(uint32_t) * n);
        if (!perm) { free(keys); return NULL; }
        for (uint64_t i = 0; i < n; i++) perm[i] = (uint32_t)i;
        xrng pr; xr_seed(&pr, sub_seed(seed, 0xFFFFFFFFULL));
        for (uint64_t i = n - 1; i > 0; i--) {
            uint64_t j = xr_below(&pr, i + 1);
            uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
        }
    }

#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t ch = 0; ch < (int64_t)nchunks; ch++) {
        xrng r; xr_seed(&r, sub_seed(seed, (uint64_t)ch));
        uint64_t lo = (uint64_t)ch * RMAT_CHUNK;
        uint64_t hi = lo + RMAT_CHUNK < samples ? lo + RMAT_CHUNK : samples;
        for (uint64_t s = lo; s < hi; s++) {
            uint64_t u = 0, v = 0;
            uint64_t word = 0;
            for (int lev = 0; lev < scale; lev++) {
                uint32_t x;
                if ((lev & 1) == 0) { word = xr_next(&r); x = (uint32_t)(word >> 32); }
                else x = (uint32_t)word;
                uint64_t bu, bv;
                if (x < ta) { bu = 0; bv = 0; }
                else if (x < tb) { bu = 0; bv = 1; }
                else if (x < tc) { bu = 1; bv = 0; }
                else { bu = 1; bv = 1; }
                u = (u << 1) | bu;
                v = (v << 1) | bv;
            }
            if (perm) { u = perm[u]; v = perm[v]; }
            keys[s] = (u << 32) | v;
        }
    }
    free(perm);
    *m_out = sort_unique_no_self(keys, samples);
    return keys;
}

/*
 * Road-like grid: rows x cols vertices (id = r * cols + c), an arc to each of the up
 * to four grid neighbours, plus round(longrange_frac * grid arcs) uniformly random
 * pairs u != v.  Duplicates are removed.  Output as for synth_rmat.
 */
uint64_t *synth_grid(uint32_t rows, uint32_t cols, double longrange_frac, uint64_t seed,
                     uint64_t *m_out)
{
    uint64_t n = (uint64_t)rows * cols;
    uint64_t grid_arcs = 2ULL * rows * (cols ? cols - 1 : 0) + 2ULL * cols * (rows ? rows - 1 : 0);
    uint64_t extra = (uint64_t)nearbyint(longrange_frac * (double)grid_arcs);
    uint64_t total = grid_arcs + extra;
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (total ? total : 1));
    if (!keys) return NULL;
    uint64_t w = 0;
    for (uint64_t r = 0; r < rows; r++) {
        for (uint64_t c = 0; c < cols; c++) {
            uint64_t u = r * cols + c;
            if (r > 0) keys[w++] = (u << 32) | (u - cols);
            if (r + 1 < rows) keys[w++] = (u << 32) | (u + cols);
            if (c > 0) keys[w++] = (u << 32) | (u - 1);
            if (c + 1 < cols) keys[w++] = (u << 32) | (u + 1);
        }
    }
    uint64_t nchunks = (extra + RMAT_CHUNK - 1) / RMAT_CHUNK;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t ch = 0; ch < (int64_t)nchunks; ch++) {
        xrng r; xr_seed(&r, sub_seed(seed, (uint64_t)ch));
        uint64_t lo = (uint64_t)ch * RMAT_CHUNK;
        uint64_t hi = lo + RMAT_CHUNK < extra ? lo + RMAT_CHUNK : extra;
        for (uint64_t s = lo; s < hi; s++) {
            uint64_t u, v;
            do { u = xr_below(&r, n); v = xr_below(&r, n); } while (u == v);
            keys[grid_arcs + s] = (u << 32) | v;
        }
    }
    *m_out = sort_unique_no_self(keys, total);
    return keys;
}

/*
 * Low-degree stand-in for the protein k-mer graphs (Table 1: 171-214 M vertices, average
 * degree 3.1 with self-loops): a seeded uniform permutation pi of the n vertices is cut
 * into chains (unitigs) that link pi[i] and pi[i+1] in both directions; the link after
 * position i is cut with probability 1 / mean_chain, and a cut instead joins pi[i] to a
 * vertex 2..65 places further along pi (both directions), as a junction does.  A further
 * fraction branch_frac of positions gets such a symmetric arc as well.  The result is one
 * long component with only local shortcuts (diameter of order n / 30), like a de Bruijn
 * graph's unitigs and bubbles, under a random vertex numbering.  Average out-degree about
 * 2 + 2 branch_frac.  Output as for synth_rmat.
 */
uint64_t *synth_kmer(uint32_t n, double mean_chain, double branch_frac, uint64_t seed, uint64_t *m_out)
{
    if (n < 2 || mean_chain < 1.0) { *m_out = 0; return (uint64_t *)malloc(sizeof(uint64_t)); }
    uint32_t *pi = (uint32_t *)malloc(sizeof(uint32_t) * n);
    if (!pi) return NULL;
    for (uint32_t i = 0; i < n; i++) pi[i] = i;
    xrng r; xr_seed(&r, sub_seed(seed, 0x6b6d6572ULL));
    for (uint64_t i = n; i > 1; i--) {
        uint64_t j = xr_below(&r, i);
        uint32_t t = pi[i - 1]; pi[i - 1] = pi[j]; pi[j] = t;
    }
    /* two arcs per position for the chain link or junction, two more for a branch */
    uint64_t cap = 4ULL * n;
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * cap);
    if (!keys) { free(pi); return NULL; }
    const uint64_t none = ~0ULL;
    const uint64_t cut = (uint64_t)((double)UINT32_MAX / mean_chain);
    const uint64_t br = (uint64_t)(branch_frac * (double)UINT32_MAX);
    uint64_t nchunks = ((uint64_t)n + RMAT_CHUNK - 1) / RMAT_CHUNK;
#pragma omp parallel for schedule(static)
    for (int64_t ch = 0; ch < (int64_t)nchunks; ch++) {
        xrng q; xr_seed(&q, sub_seed(seed, (uint64_t)ch));
        uint64_t lo = (uint64_t)ch * RMAT_CHUNK;
        uint64_t hi = lo + RMAT_CHUNK < n ? lo + RMAT_CHUNK : n;
        for (uint64_t i = lo; i < hi; i++) {
            uint64_t u = pi[i], *o = keys + 4 * i;
            o[0] = o[1] = o[2] = o[3] = none;
            if (i + 1 < n) {
                uint64_t j = (xr_next(&q) & 0xFFFFFFFFULL) < cut ? i + 2 + xr_below(&q, 64) : i + 1;
                if (j < n) {
                    uint64_t w = pi[j];
                    o[0] = (u << 32) | w;
                    o[1] = (w << 32) | u;
                }
            }
            if ((xr_next(&q) & 0xFFFFFFFFULL) < br) {
                uint64_t j = i + 2 + xr_below(&q, 64);
                if (j < n) {
                    uint64_t w = pi[j];
                    o[2] = (u << 32) | w;
                    o[3] = (w << 32) | u;
                }
            }
        }
    }
    free(pi);
    uint64_t w = 0;
    for (uint64_t i = 0; i < cap; i++) if (keys[i] != none) keys[w++] = keys[i];
    *m_out = sort_unique_no_self(keys, w);
    return keys;
}

void synth_free(void *p) { free(p); }

/* Split sorted keys into source and target arrays. */
void synth_keys_split(const uint64_t *keys, uint64_t m, uint32_t *src, uint32_t *dst)
{
    for (uint64_t i = 0; i < m; i++) {
        src[i] = (uint32_t)(keys[i] >> 32);
        dst[i] = (uint32_t)keys[i];
    }
}

/* ------------------------------------------------------------ batch stream ---- */

/*
 * A stream of random batch updates against an evolving edge set (Section 5.1.4):
 * batch t of fraction f holds k = max(1, round(f * base_m)) edges, of which
 * round(ins_share * k) are insertions of uniformly random pairs u != v absent from the
 * current set (and distinct within the batch) and the rest deletions of distinct
 * current edges chosen uniformly without replacement.  base_m is the edge count of the
 * original graph.  Rounding is half-to-even.  After each batch the stream applies it to
 * its own copy of the edge set, so the next batch is drawn against the updated graph.
 * The stream's seed for batch t is sub_seed(seed, t).
 */
typedef struct {
    uint32_t n;
    uint64_t base_m;
    uint64_t seed;
    uint64_t t;
    uint64_t m;      /* current edges */
    uint64_t cap;
    uint64_t *keys;  /* sorted unique, no self pairs */
} synth_stream;

synth_stream *synth_stream_create(uint32_t n, const uint64_t *keys, uint64_t m, uint64_t base_m,
                                  uint64_t seed)
{
    synth_stream *s = (synth_stream *)calloc(1, sizeof(synth_stream));
    if (!s) return NULL;
    s->n = n; s->base_m = base_m; s->seed = seed; s->t = 0; s->m = m;
    s->cap = m + 1024;
    s->keys = (uint64_t *)malloc(sizeof(uint64_t) * s->cap);
    if (!s->keys) { free(s); return NULL; }
    memcpy(s->keys, keys, sizeof(uint64_t) * m);
    return s;
}

void synth_stream_destroy(synth_stream *s)
{
    if (!s) return;
    free(s->keys);
    free(s);
}

uint64_t synth_stream_m(const synth_stream *s) { return s->m; }
const uint64_t *synth_stream_keys(const synth_stream *s) { return s->keys; }

static void shuffle_u64(uint64_t *a, uint64_t n, xrng *r)
{
    for (uint64_t i = n; i > 1; i--) {
        uint64_t j = xr_below(r, i);
        uint64_t t = a[i - 1]; a[i - 1] = a[j]; a[j] = t;
    }
}

static int cmp_u64(const void *x, const void *y)
{
    uint64_t a = *(const uint64_t *)x, b = *(const uint64_t *)y;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* Sizes of the next batch of fraction `frac`. */
void synth_batch_sizes(uint64_t base_m, double frac, double ins_share, uint64_t *k_ins,
                       uint64_t *k_del)
{
    double kd = nearbyint(frac * (double)base_m);
    uint64_t k = kd < 1.0 ? 1 : (uint64_t)kd;
    uint64_t ki = (uint64_t)nearbyint(ins_share * (double)k);
    if (ki > k) ki = k;
    *k_ins = ki;
    *k_del = k - ki;
}

/*
 * Draws the next batch.  Outputs (caller-allocated, sizes from synth_batch_sizes):
 * del_src/del_dst [k_del], ins_src/ins_dst [k_ins], each in a seeded random order.
 * If `apply` is set the stream's edge set advances to (E \ D) U I.
 * Returns 0, or -1 if the request cannot be met (too few edges / absent pairs).
 */
int synth_stream_next(synth_stream *s, double frac, double ins_share, int apply,
                      uint32_t *del_src, uint32_t *del_dst, uint32_t *ins_src, uint32_t *ins_dst)
{
    uint64_t k_ins, k_del;
    synth_batch_sizes(s->base_m, frac, ins_share, &k_ins, &k_del);
    if (k_del > s->m) return -1;
    uint64_t n = s->n;
    if (n < 2 || (double)k_ins + (double)s->m > (double)n * (double)(n - 1)) return -1;
    xrng r; xr_seed(&r, sub_seed(s->seed, s->t));
    s->t++;

    /* deletions: distinct indices into the current sorted key array */
    uint64_t *didx = (uint64_t *)malloc(sizeof(uint64_t) * (k_del + 1));
    uint64_t have = 0;
    while (have < k_del) {
        for (uint64_t i = have; i < k_del; i++) didx[i] = xr_below(&r, s->m);
        qsort(didx, k_del, sizeof(uint64_t), cmp_u64);
        uint64_t w = 0;
        for (uint64_t i = 0; i < k_del; i++) if (w == 0 || didx[w - 1] != didx[i]) didx[w++] = didx[i];
        have = w;
    }
    /* insertions: uniform pairs u != v, absent from E, distinct within the batch */
    uint64_t *ikeys = (uint64_t *)malloc(sizeof(uint64_t) * (k_ins + 1));
    have = 0;
    while (have < k_ins) {
        for (uint64_t i = have; i < k_ins; i++) {
            uint64_t u, v, key;
            do {
                u = xr_below(&r, n);
                v = xr_below(&r, n);
                key = (u << 32) | v;
            } while (u == v || contains_u64(s->keys, (int64_t)s->m, key));
            ikeys[i] = key;
        }
        qsort(ikeys, k_ins, sizeof(uint64_t), cmp_u64);
        uint64_t w = 0;
        for (uint64_t i = 0; i < k_ins; i++) if (w == 0 || ikeys[w - 1] != ikeys[i]) ikeys[w++] = ikeys[i];
        have = w;
    }
    /* outputs in a seeded random order */
    uint64_t *dkeys = (uint64_t *)malloc(sizeof(uint64_t) * (k_del + 1));
    for (uint64_t i = 0; i < k_del; i++) dkeys[i] = s->keys[didx[i]];
    uint64_t *dout = (uint64_t *)malloc(sizeof(uint64_t) * (k_del + 1));
    uint64_t *iout = (uint64_t *)malloc(sizeof(uint64_t) * (k_ins + 1));
    memcpy(dout, dkeys, sizeof(uint64_t) * k_del);
    memcpy(iout, ikeys, sizeof(uint64_t) * k_ins);
    shuffle_u64(dout, k_del, &r);
    shuffle_u64(iout, k_ins, &r);
    for (uint64_t i = 0; i < k_del; i++) { del_src[i] = (uint32_t)(dout[i] >> 32); del_dst[i] = (uint32_t)dout[i]; }
    for (uint64_t i = 0; i < k_ins; i++) { ins_src[i] = (uint32_t)(iout[i] >> 32); ins_dst[i] = (uint32_t)iout[i]; }
    free(dout); free(iout);

    if (apply) {
        /* remove deleted indices (sorted), then merge sorted insertions */
        uint64_t newm = s->m - k_del + k_ins;
        uint64_t *nk = (uint64_t *)malloc(sizeof(uint64_t) * (newm + 1024));
        uint64_t i = 0, j = 0, d = 0, w = 0;
        while (i < s->m || j < k_ins) {
            if (i < s->m && d < k_del && didx[d] == i) { i++; d++; continue; }
            if (j >= k_ins || (i < s->m && s->keys[i] < ikeys[j])) nk[w++] = s->keys[i++];
            else nk[w++] = ikeys[j++];
        }
        free(s->keys);
        s->keys = nk;
        s->m = w;
        s->cap = newm + 1024;
    }
    free(didx); free(ikeys); free(dkeys);
    return 0;
}

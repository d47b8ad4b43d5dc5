/*
 * Seeded synthetic input generators for the LLP problems.
 *
 * This module only draws random inputs and lays them out (edge lists -> CSR by a
 * stable counting sort).  It holds none of the arithmetic of the method: no
 * relaxation, no proposal, no DP, no closure.  Both the oracle and the CUDA path
 * consume what it writes.
 *
 * Random numbers:
 *   - SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
 *     generators", OOPSLA 2014) expands a 64-bit seed into generator state;
 *   - xoshiro256** (Blackman and Vigna, "Scrambled linear pseudorandom number
 *     generators", ACM TOMS 2021) is the stream generator;
 *   - bounded integers use Lemire's multiply-shift rejection method ("Fast random
 *     integer generation in an interval", ACM TOMACS 2019), so [lo,hi] draws are
 *     unbiased;
 *   - Poisson variates use Knuth's product-of-uniforms method (TAOCP vol. 2,
 *     3.4.1), fine for the small means used here.
 * Every stream is keyed by (seed, stream id) so that independent parts of one
 * instance never share a stream.  Large edge lists are drawn in fixed blocks of
 * 2^20 edges, each block with its own stream, so the output does not depend on
 * the number of host threads used.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static void rng_init(rng_t *r, uint64_t seed, uint64_t stream) {
    uint64_t x = seed ^ (stream * 0xd1342543de82ef95ULL + 0x632be59bd9b4e019ULL);
    for (int i = 0; i < 4; i++) r->s[i] = splitmix64_next(&x);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_u64(rng_t *r) {
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

/* uniform in [0, range), range >= 1 (Lemire 2019) */
static inline uint64_t rng_below(rng_t *r, uint64_t range) {
    unsigned __int128 m = (unsigned __int128)rng_u64(r) * range;
    uint64_t lo = (uint64_t)m;
    if (lo < range) {
        uint64_t thresh = (0 - range) % range;
        while (lo < thresh) {
            m = (unsigned __int128)rng_u64(r) * range;
            lo = (uint64_t)m;
        }
    }
    return (uint64_t)(m >> 64);
}

/* uniform in [lo, hi] inclusive */
static inline int64_t rng_range(rng_t *r, int64_t lo, int64_t hi) {
    return lo + (int64_t)rng_below(r, (uint64_t)(hi - lo) + 1);
}

static inline double rng_unit(rng_t *r) { return (double)(rng_u64(r) >> 11) * (1.0 / 9007199254740992.0); }

static int rng_poisson(rng_t *r, double lambda) {
    double L = exp(-lambda), p = 1.0;
    int k = 0;
    do { k++; p *= rng_unit(r); } while (p > L);
    return k - 1;
}

/* --------------------------------------------------------------- generic */

void synth_fill_u64(int64_t n, uint64_t seed, uint64_t *out) {
    const int64_t B = 1 << 20;
    int64_t nb = (n + B - 1) / B;
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nb; b++) {
        rng_t r;
        rng_init(&r, seed, 1000 + (uint64_t)b);
        int64_t e1 = (b + 1) * B < n ? (b + 1) * B : n;
        for (int64_t i = b * B; i < e1; i++) out[i] = rng_u64(&r);
    }
}

/* values uniform in [lo, hi], int32 */
void synth_fill_i32(int64_t n, int32_t lo, int32_t hi, uint64_t seed, uint64_t stream, int32_t *out) {
    const int64_t B = 1 << 20;
    int64_t nb = (n + B - 1) / B;
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nb; b++) {
        rng_t r;
        rng_init(&r, seed, stream * 65536 + (uint64_t)b);
        int64_t e1 = (b + 1) * B < n ? (b + 1) * B : n;
        for (int64_t i = b * B; i < e1; i++) out[i] = (int32_t)rng_range(&r, lo, hi);
    }
}

/* uniform random permutation of 0..n-1 (Fisher-Yates) */
static void perm(rng_t *r, int32_t n, int32_t *p) {
    for (int32_t i = 0; i < n; i++) p[i] = i;
    for (int32_t i = n - 1; i > 0; i--) {
        int32_t j = (int32_t)rng_below(r, (uint64_t)i + 1);
        int32_t t = p[i]; p[i] = p[j]; p[j] = t;
    }
}

/* ------------------------------------------------------------ edge lists */

/* Erdos-Renyi G(n, M): M ordered pairs drawn i.i.d. uniform, duplicates and
 * self-loops kept; weights uniform in [wlo, whi]. */
void synth_er_edges(int32_t n, int64_t m, uint32_t wlo, uint32_t whi, uint64_t seed,
                    int32_t *src, int32_t *dst, uint32_t *w) {
    const int64_t B = 1 << 20;
    int64_t nb = (m + B - 1) / B;
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nb; b++) {
        rng_t r, rw;
        rng_init(&r, seed, 1 + 2 * (uint64_t)b);
        rng_init(&rw, seed, 2 + 2 * (uint64_t)b + (1ULL << 40));
        int64_t e1 = (b + 1) * B < m ? (b + 1) * B : m;
        for (int64_t e = b * B; e < e1; e++) {
            src[e] = (int32_t)rng_below(&r, (uint64_t)n);
            dst[e] = (int32_t)rng_below(&r, (uint64_t)n);
        }
        for (int64_t e = b * B; e < e1; e++) w[e] = (uint32_t)rng_range(&rw, wlo, whi);
    }
}

/* R-MAT (Chakrabarti, Zhan, Faloutsos 2004): per edge, one quadrant per bit
 * level with probabilities (a, b, c, 1-a-b-c), no noise; then a seeded random
 * relabelling of the vertices (as in the Graph500 generator) so that hubs are
 * spread over the id range.  Self-loops and duplicates kept.  Weights are drawn
 * after the edges from their own streams. */
void synth_rmat_edges(int32_t scale, int64_t m, double a, double b, double c,
                      uint32_t wlo, uint32_t whi, uint64_t seed,
                      int32_t *src, int32_t *dst, uint32_t *w) {
    const int64_t B = 1 << 20;
    int64_t nb = (m + B - 1) / B;
    const uint64_t ta = (uint64_t)(a * 4294967296.0);
    const uint64_t tb = (uint64_t)((a + b) * 4294967296.0);
    const uint64_t tc = (uint64_t)((a + b + c) * 4294967296.0);
    int32_t n = (int32_t)(1u << scale);
#pragma omp parallel for schedule(static)
    for (int64_t blk = 0; blk < nb; blk++) {
        rng_t r;
        rng_init(&r, seed, 1 + (uint64_t)blk);
        int64_t e1 = (blk + 1) * B < m ? (blk + 1) * B : m;
        for (int64_t e = blk * B; e < e1; e++) {
            uint32_t u = 0, v = 0;
            uint64_t bits = 0;
            int have = 0;
            for (int lvl = 0; lvl < scale; lvl++) {
                if (!have) { bits = rng_u64(&r); have = 2; }
                uint64_t x = bits & 0xffffffffULL;
                bits >>= 32;
                have--;
                uint32_t ub, vb;
                if (x < ta) { ub = 0; vb = 0; }
                else if (x < tb) { ub = 0; vb = 1; }
                else if (x < tc) { ub = 1; vb = 0; }
                else { ub = 1; vb = 1; }
                u = (u << 1) | ub;
                v = (v << 1) | vb;
            }
            src[e] = (int32_t)u;
            dst[e] = (int32_t)v;
        }
    }
    /* relabel */
    int32_t *p = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    rng_t rp;
    rng_init(&rp, seed, 0x5eed0000ULL);
    perm(&rp, n, p);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; e++) {
        src[e] = p[src[e]];
        dst[e] = p[dst[e]];
    }
    free(p);
#pragma omp parallel for schedule(static)
    for (int64_t blk = 0; blk < nb; blk++) {
        rng_t rw;
        rng_init(&rw, seed, (1ULL << 40) + (uint64_t)blk);
        int64_t e1 = (blk + 1) * B < m ? (blk + 1) * B : m;
        for (int64_t e = blk * B; e < e1; e++) w[e] = (uint32_t)rng_range(&rw, wlo, whi);
    }
}

/* 2-D rows x cols 4-neighbour grid; vertex id r*cols+c; both arc directions,
 * each arc with its own weight uniform in [wlo, whi].  Arcs are emitted in
 * source order, neighbours in the order up, down, left, right. */
int64_t synth_grid_edges(int32_t rows, int32_t cols, uint32_t wlo, uint32_t whi, uint64_t seed,
                         int32_t *src, int32_t *dst, uint32_t *w) {
    rng_t r;
    rng_init(&r, seed, 7);
    int64_t e = 0;
    for (int32_t i = 0; i < rows; i++)
        for (int32_t j = 0; j < cols; j++) {
            int32_t u = i * cols + j;
            const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
            for (int k = 0; k < 4; k++) {
                int32_t ii = i + di[k], jj = j + dj[k];
                if (ii < 0 || ii >= rows || jj < 0 || jj >= cols) continue;
                src[e] = u;
                dst[e] = ii * cols + jj;
                w[e] = (uint32_t)rng_range(&r, wlo, whi);
                e++;
            }
        }
    return e;
}

/* Random DAG on n vertices: each pair i<j is an arc i->j with probability
 * pnum/pden.  Writes at most cap arcs; returns the arc count (or -1 if cap
 * was too small). */
int64_t synth_random_dag_edges(int32_t n, uint64_t pnum, uint64_t pden, uint64_t seed,
                               int64_t cap, int32_t *src, int32_t *dst) {
    rng_t r;
    rng_init(&r, seed, 11);
    int64_t e = 0;
    for (int32_t i = 0; i < n; i++)
        for (int32_t j = i + 1; j < n; j++)
            if (rng_below(&r, pden) < pnum) {
                if (e >= cap) return -1;
                src[e] = i;
                dst[e] = j;
                e++;
            }
    return e;
}

/* Job DAG: for job j draw k ~ Poisson(lambda) and choose min(k, n-1-j)
 * distinct successors uniformly from {j+1, ..., n-1} (rejection against the
 * already chosen ones); durations uniform in [tlo, thi].  Arcs in source order.
 * Returns the arc count, or -1 if cap is too small. */
int64_t synth_job_dag(int32_t n, double lambda, int32_t tlo, int32_t thi, uint64_t seed, int64_t cap,
                      int32_t *src, int32_t *dst, int32_t *duration) {
    rng_t r, rt;
    rng_init(&r, seed, 13);
    rng_init(&rt, seed, 17);
    int64_t e = 0;
    int32_t chosen[64];
    for (int32_t j = 0; j < n; j++) {
        duration[j] = (int32_t)rng_range(&rt, tlo, thi);
        int k = rng_poisson(&r, lambda);
        int32_t avail = n - 1 - j;
        if (k > avail) k = avail;
        if (k > 64) k = 64;
        int got = 0;
        while (got < k) {
            int32_t t = j + 1 + (int32_t)rng_below(&r, (uint64_t)avail);
            int dup = 0;
            for (int q = 0; q < got; q++) dup |= (chosen[q] == t);
            if (dup) continue;
            chosen[got++] = t;
        }
        for (int q = 0; q < got; q++) {
            if (e >= cap) return -1;
            src[e] = j;
            dst[e] = chosen[q];
            e++;
        }
    }
    return e;
}

/* ------------------------------------------------------------------- CSR */

/* Stable counting sort of arcs by source: offsets[n+1] (int64), and the arc
 * payloads permuted accordingly (w may be NULL).  Arc order inside a row is
 * the order of the input list. */
void synth_csr_from_edges(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                          const uint32_t *w, int64_t *offsets, int32_t *indices, uint32_t *weights) {
    memset(offsets, 0, sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t e = 0; e < m; e++) offsets[src[e] + 1]++;
    for (int32_t v = 0; v < n; v++) offsets[v + 1] += offsets[v];
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    memcpy(pos, offsets, sizeof(int64_t) * (size_t)n);
    for (int64_t e = 0; e < m; e++) {
        int64_t p = pos[src[e]]++;
        indices[p] = dst[e];
        if (w && weights) weights[p] = w[e];
    }
    free(pos);
}

/* ---------------------------------------------------------- preferences */

/* Random stable-marriage instance: men_pref[m*n+k] = k-th woman of man m
 * (independent Fisher-Yates permutations); women_rank[w*n+m] = rank of man m
 * for woman w (0 = most preferred), the inverse of an independent permutation.
 * If shared_men_order is non-zero, all men share one preference order
 * (the adversarial instance). */
void synth_marriage(int32_t n, uint64_t seed, int shared_men_order, int32_t *men_pref, int32_t *women_rank) {
#pragma omp parallel
    {
        int32_t *p = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
#pragma omp for schedule(static)
        for (int32_t m = 0; m < n; m++) {
            rng_t r;
            rng_init(&r, seed, shared_men_order ? 100 : 100 + (uint64_t)m);
            perm(&r, n, men_pref + (size_t)m * n);
        }
#pragma omp for schedule(static)
        for (int32_t w = 0; w < n; w++) {
            rng_t r;
            rng_init(&r, seed, (1ULL << 32) + (uint64_t)w);
            perm(&r, n, p);
            int32_t *row = women_rank + (size_t)w * n;
            for (int32_t k = 0; k < n; k++) row[p[k]] = k;
        }
        free(p);
    }
}

/* ------------------------------------------------------- batched configs */

/* Sizes of a batch: count values uniform in [lo, hi] from stream `stream`. */
void synth_sizes(int32_t count, int64_t lo, int64_t hi, uint64_t seed, uint64_t stream, int64_t *out) {
    rng_t r;
    rng_init(&r, seed, stream);
    for (int32_t i = 0; i < count; i++) out[i] = rng_range(&r, lo, hi);
}

/* One 0-1 knapsack instance: weights uniform in [1, max(1, W/4)], values in
 * [vlo, vhi]. */
void synth_knapsack(int32_t n, int32_t W, int32_t vlo, int32_t vhi, uint64_t seed, uint64_t stream,
                    int32_t *w, int32_t *v) {
    rng_t r;
    rng_init(&r, seed, stream);
    int32_t wmax = W / 4 > 1 ? W / 4 : 1;
    for (int32_t i = 0; i < n; i++) w[i] = (int32_t)rng_range(&r, 1, wmax);
    for (int32_t i = 0; i < n; i++) v[i] = (int32_t)rng_range(&r, vlo, vhi);
}

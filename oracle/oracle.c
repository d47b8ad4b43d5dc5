/*
 * LLP oracle: plain, sequential, obviously-correct CPU implementations of what
 * each LLP sweep converges to.  TEST INFRASTRUCTURE ONLY: only tests, the smoke
 * check and the benchmark's CPU-baseline leg may call it; the product path never
 * links or loads it.  It shares no code, header or table with the CUDA path.
 *
 * Every LLP problem of the paper reaches (Algorithm LLP, Sec. 3) the least
 * vector satisfying its lattice-linear predicate.  For each problem that least
 * vector has a classical, plain definition, and this file computes that
 * definition with the textbook sequential algorithm:
 *
 *   SSSP      d(s)=0, d(v)=min path weight (Sec. 4.1 problem definition);
 *             Dijkstra, binary heap, lazy deletion.
 *   BFS       hop level from the source (Sec. 4.2); FIFO queue BFS.
 *   Marriage  man-optimal stable matching, the fixed point LLP reaches
 *             (Sec. 4.3); man-proposing Gale-Shapley with a free-man stack.
 *   Jobs      G[j] = t_j + max over predecessors of G[p], 0 for none
 *             (Sec. 4.4 formulation); Kahn topological order, longest path.
 *   Reduce    sum of the inputs modulo 2^64 (Sec. 4.5); sequential loop.
 *   Closure   R[u][v] = 1 iff a directed path of length >= 1 exists (Sec. 4.6);
 *             Warshall on bit-packed rows.
 *   Knapsack  dp[k][c] = max(dp[k-1][c], v_k + dp[k-1][c-w_k]) (Sec. 4.7);
 *             the row-by-row DP table.
 *
 * Encodings (readings where the paper is silent): "infinity" of SSSP/BFS is
 * 0xFFFFFFFF; path sums are formed in 64 bits and a finite distance that does
 * not fit below 0xFFFFFFFF is reported as overflow.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_INF 0xFFFFFFFFu

enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_OVERFLOW = 6, OR_ERR_CYCLE = 8, OR_ERR_INFEASIBLE = 5, OR_ERR_NOMEM = 9 };

/* ------------------------------------------------------------- Dijkstra */

typedef struct { uint64_t key; int32_t v; } heap_item;

static void heap_push(heap_item *h, int64_t *sz, uint64_t key, int32_t v) {
    int64_t i = (*sz)++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h[p].key <= key) break;
        h[i] = h[p];
        i = p;
    }
    h[i].key = key;
    h[i].v = v;
}

static heap_item heap_pop(heap_item *h, int64_t *sz) {
    heap_item top = h[0];
    heap_item last = h[--(*sz)];
    int64_t i = 0, n = *sz;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= n) break;
        if (c + 1 < n && h[c + 1].key < h[c].key) c++;
        if (h[c].key >= last.key) break;
        h[i] = h[c];
        i = c;
    }
    if (n > 0) h[i] = last;
    return top;
}

/* Single-source shortest paths over the out-arcs of a CSR graph (offsets are
 * int64[n+1], indices int32[m], weights uint32[m]; weights==NULL means every
 * weight is 1).  dist[v] = 0xFFFFFFFF when v is unreachable. */
int oracle_dijkstra(int32_t n, const int64_t *offsets, const int32_t *indices, const uint32_t *weights,
                    int32_t source, uint32_t *dist) {
    if (n < 1 || source < 0 || source >= n) return OR_ERR_ARG;
    uint64_t *d = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    char *done = (char *)calloc((size_t)n, 1);
    int64_t m = offsets[n];
    heap_item *h = (heap_item *)malloc(sizeof(heap_item) * (size_t)(m + 1));
    if (!d || !done || !h) { free(d); free(done); free(h); return OR_ERR_NOMEM; }
    for (int32_t v = 0; v < n; v++) d[v] = UINT64_MAX;
    int64_t sz = 0;
    d[source] = 0;
    heap_push(h, &sz, 0, source);
    while (sz > 0) {
        heap_item it = heap_pop(h, &sz);
        int32_t u = it.v;
        if (done[u]) continue;
        done[u] = 1;
        for (int64_t e = offsets[u]; e < offsets[u + 1]; e++) {
            int32_t v = indices[e];
            uint64_t nd = d[u] + (weights ? weights[e] : 1u);
            if (nd < d[v]) {
                d[v] = nd;
                heap_push(h, &sz, nd, v);
            }
        }
    }
    int rc = OR_OK;
    for (int32_t v = 0; v < n; v++) {
        if (d[v] == UINT64_MAX) dist[v] = ORACLE_INF;
        else if (d[v] >= ORACLE_INF) { dist[v] = ORACLE_INF; rc = OR_ERR_OVERFLOW; }
        else dist[v] = (uint32_t)d[v];
    }
    free(d); free(done); free(h);
    return rc;
}

/* ------------------------------------------------------------------ BFS */

int oracle_bfs(int32_t n, const int64_t *offsets, const int32_t *indices, int32_t source, uint32_t *level) {
    if (n < 1 || source < 0 || source >= n) return OR_ERR_ARG;
    int32_t *q = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!q) return OR_ERR_NOMEM;
    for (int32_t v = 0; v < n; v++) level[v] = ORACLE_INF;
    int64_t head = 0, tail = 0;
    level[source] = 0;
    q[tail++] = source;
    while (head < tail) {
        int32_t u = q[head++];
        for (int64_t e = offsets[u]; e < offsets[u + 1]; e++) {
            int32_t v = indices[e];
            if (level[v] == ORACLE_INF) {
                level[v] = level[u] + 1;
                q[tail++] = v;
            }
        }
    }
    free(q);
    return OR_OK;
}

/* -------------------------------------------------------- Transpose
 * In-arc CSR of a graph (input of the pull form of the BFS predicate,
 * Sec. 4.2, which reads in-neighbours): in_offsets[v] = number of arcs whose
 * target is below v; row v lists the sources of the arcs into v, in the order
 * the arcs appear in the out-arc CSR (a stable counting sort by target).
 * in_weights (may be NULL) carries each arc's weight along. */
int oracle_csr_transpose(int32_t n, const int64_t *offsets, const int32_t *indices, const uint32_t *weights,
                         int64_t *in_offsets, int32_t *in_indices, uint32_t *in_weights) {
    if (n < 1) return OR_ERR_ARG;
    int64_t m = offsets[n];
    for (int32_t v = 0; v <= n; v++) in_offsets[v] = 0;
    for (int64_t e = 0; e < m; e++) {
        if (indices[e] < 0 || indices[e] >= n) return OR_ERR_ARG;
        in_offsets[indices[e] + 1]++;
    }
    for (int32_t v = 0; v < n; v++) in_offsets[v + 1] += in_offsets[v];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!fill) return OR_ERR_NOMEM;
    for (int32_t v = 0; v < n; v++) fill[v] = in_offsets[v];
    for (int32_t u = 0; u < n; u++) {
        for (int64_t e = offsets[u]; e < offsets[u + 1]; e++) {
            int64_t pos = fill[indices[e]]++;
            in_indices[pos] = u;
            if (in_weights) in_weights[pos] = weights[e];
        }
    }
    free(fill);
    return OR_OK;
}

/* ------------------------------------------------------- Gale-Shapley */

/* men_pref[m*n+k] = k-th most preferred woman of man m;
 * women_rank[w*n+m] = rank of man m in woman w's list (0 = most preferred).
 * Outputs: wife[m], husband[w] (may be NULL), next[m] = index into m's list of
 * his final partner (the LLP state G[m]; may be NULL).  Returns the number of
 * proposals made via *proposals (may be NULL). */
int oracle_gale_shapley(int32_t n, const int32_t *men_pref, const int32_t *women_rank,
                        int32_t *wife, int32_t *husband, int32_t *next, int64_t *proposals) {
    if (n < 1) return OR_ERR_ARG;
    int32_t *idx = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    int32_t *hus = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!idx || !hus || !stack) { free(idx); free(hus); free(stack); return OR_ERR_NOMEM; }
    for (int32_t w = 0; w < n; w++) hus[w] = -1;
    int32_t top = 0;
    for (int32_t m = n - 1; m >= 0; m--) stack[top++] = m;
    int64_t props = 0;
    int rc = OR_OK;
    while (top > 0) {
        int32_t m = stack[--top];
        if (idx[m] >= n) { rc = OR_ERR_INFEASIBLE; break; }
        int32_t w = men_pref[(int64_t)m * n + idx[m]];
        props++;
        int32_t h = hus[w];
        if (h < 0) {
            hus[w] = m;
        } else if (women_rank[(int64_t)w * n + m] < women_rank[(int64_t)w * n + h]) {
            hus[w] = m;
            idx[h]++;
            stack[top++] = h;
        } else {
            idx[m]++;
            stack[top++] = m;
        }
    }
    if (rc == OR_OK) {
        for (int32_t w = 0; w < n; w++) {
            if (husband) husband[w] = hus[w];
            if (hus[w] >= 0) wife[hus[w]] = w;
        }
        if (next) memcpy(next, idx, sizeof(int32_t) * (size_t)n);
    }
    if (proposals) *proposals = props;
    free(idx); free(hus); free(stack);
    return rc;
}

/* ------------------------------------------------------------ knapsack */

/* 0-1 knapsack DP over items in the given order with capacity constraint
 * "<= W": dp[0][c] = 0; dp[k][c] = max(dp[k-1][c], v_k + dp[k-1][c-w_k]) when
 * w_k <= c.  Rows k-1 and k are kept (the table is filled row by row).
 * Writes the last row to row_out[0..W] if non-NULL; returns dp[n][W] in *best. */
int oracle_knapsack(int32_t n, const int32_t *w, const int32_t *v, int32_t W, int32_t *best, int32_t *row_out) {
    if (n < 0 || W < 0) return OR_ERR_ARG;
    int64_t *prev = (int64_t *)calloc((size_t)W + 1, sizeof(int64_t));
    int64_t *cur = (int64_t *)calloc((size_t)W + 1, sizeof(int64_t));
    if (!prev || !cur) { free(prev); free(cur); return OR_ERR_NOMEM; }
    for (int32_t k = 0; k < n; k++) {
        for (int32_t c = 0; c <= W; c++) {
            int64_t keep = prev[c];
            int64_t take = (w[k] <= c) ? (int64_t)v[k] + prev[c - w[k]] : INT64_MIN;
            cur[c] = keep > take ? keep : take;
        }
        int64_t *t = prev; prev = cur; cur = t;
    }
    int rc = OR_OK;
    if (prev[W] > INT32_MAX) rc = OR_ERR_OVERFLOW;
    *best = (int32_t)prev[W];
    if (row_out)
        for (int32_t c = 0; c <= W; c++) row_out[c] = (int32_t)prev[c];
    free(prev); free(cur);
    return rc;
}

/* ---------------------------------------------------- transitive closure */

/* reach has n rows of W = ceil(n/32) uint32 words; bit (v & 31) of word
 * reach[u*W + v/32] (least significant bit first) is 1 iff v is reachable from
 * u by a path of one or more arcs.  Warshall: R := adjacency; for every k, every
 * row i containing k absorbs row k. */
int oracle_warshall(int32_t n, const int64_t *offsets, const int32_t *indices, uint32_t *reach) {
    if (n < 1) return OR_ERR_ARG;
    int64_t W = (n + 31) / 32;
    memset(reach, 0, sizeof(uint32_t) * (size_t)(W * n));
    for (int32_t u = 0; u < n; u++)
        for (int64_t e = offsets[u]; e < offsets[u + 1]; e++) {
            int32_t v = indices[e];
            reach[u * W + v / 32] |= 1u << (v & 31);
        }
    for (int32_t k = 0; k < n; k++) {
        const uint32_t *rk = reach + k * W;
        for (int32_t i = 0; i < n; i++) {
            uint32_t *ri = reach + i * W;
            if (ri[k / 32] & (1u << (k & 31)))
                for (int64_t x = 0; x < W; x++) ri[x] |= rk[x];
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------- job scheduling */

/* Successor CSR (succ_offsets int64[n+1], succ_indices int32[m]); durations
 * t_j >= 0.  completion[j] = t_j + max over predecessors p of completion[p]
 * (0 for no predecessors), computed in Kahn topological order.  Returns
 * OR_ERR_CYCLE if the graph is not acyclic. */
int oracle_job_schedule(int32_t n, const int32_t *duration, const int64_t *succ_offsets,
                        const int32_t *succ_indices, int32_t *completion) {
    if (n < 1) return OR_ERR_ARG;
    int32_t *indeg = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    int64_t *start = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    int32_t *q = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!indeg || !start || !q) { free(indeg); free(start); free(q); return OR_ERR_NOMEM; }
    for (int64_t e = 0; e < succ_offsets[n]; e++) indeg[succ_indices[e]]++;
    int64_t head = 0, tail = 0;
    for (int32_t j = 0; j < n; j++)
        if (indeg[j] == 0) q[tail++] = j;
    int rc = OR_OK;
    while (head < tail) {
        int32_t j = q[head++];
        int64_t c = start[j] + duration[j];
        if (c > INT32_MAX) rc = OR_ERR_OVERFLOW;
        completion[j] = (int32_t)c;
        for (int64_t e = succ_offsets[j]; e < succ_offsets[j + 1]; e++) {
            int32_t s = succ_indices[e];
            if (c > start[s]) start[s] = c;
            if (--indeg[s] == 0) q[tail++] = s;
        }
    }
    if (tail != n) rc = OR_ERR_CYCLE;
    free(indeg); free(start); free(q);
    return rc;
}

/* ----------------------------------------------------------- reduction */

uint64_t oracle_sum_u64(int64_t n, const uint64_t *x) {
    uint64_t s = 0;
    for (int64_t i = 0; i < n; i++) s += x[i];
    return s;
}

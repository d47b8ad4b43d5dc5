// Persistent forbidden/advance sweep engine for the graph problems:
// SSSP (paper Sec. 4.1) and BFS (paper Sec. 4.2).
//
// State G = dist[] (uint32, 0xFFFFFFFF = "infinity").  A vertex v is forbidden
// when some arc (u, v) offers d(u) + w(u, v) < d(v); the advance lowers d(v)
// with atomicMin, the lock-free monotone update whose requirements the paper
// lists in Sec. 3.2 (atomic, monotone, progress detection).  The predicate is
// evaluated push-style: when u is taken from the worklist, each out-arc is
// checked, and every successful advance makes v a candidate of the next sweep
// (the paper's problem-specific state selection, Sec. 3.2).
//
// One cooperative launch runs all sweeps, separated by a bounded grid barrier.
//   - stamp[v] = (sweep << 2) | class, class 0: no out-arcs (never needs a
//     visit), 1: small (out-degree <= small_max), 2: large.  v belongs to the
//     worklist of sweep k iff stamp[v] >> 2 == k; atomicMax on the stamp
//     deduplicates.
//   - small vertices are taken 32 per warp and their arcs expanded
//     edge-balanced inside the warp; large vertices are cut into chunks of
//     chunk_edges arcs, one chunk per warp, so hubs spread over the grid.
//   - sparse sweeps walk a list of small vertices (built with warp-aggregated
//     appends); dense sweeps scan every stamp instead (the paper's all-indices
//     solver) and read the CSR in vertex order.  While a sweep is dense, the
//     next one is too, and small vertices are then only stamped (no list, no
//     shared counter in the hot loop; one count per CTA at the end).
//   - with a finite bucket width delta (the paper's bucket worklist, Sec. 3.3),
//     only advances with d < current bucket bound enter the next worklist; the
//     others wait in a far list filtered when the near worklist empties.
// The run stops when no index is forbidden: both worklists are empty.
#include <algorithm>

#include "llp_common.cuh"

namespace llp {
namespace {

struct BlockCfg {
    int small_max;
    int chunk;
};
__host__ __device__ inline BlockCfg block_cfg_of(int c) {
    return c == 1 ? BlockCfg{16, 128} : (c == 3 ? BlockCfg{64, 512} : BlockCfg{32, 256});
}

constexpr int kUnroll = 4;  // arcs per lane in flight

template <typename OffT>
struct GraphArgs {
    int32_t n;
    int32_t source;
    const OffT *off;
    const int32_t *idx;
    const uint32_t *w;
    uint32_t *dist;
    uint32_t *stamp;
    int32_t *small[2];
    int2 *chunk[2];
    int2 *far[2];
    uint32_t far_cap;
    WsHeader *h;
    uint32_t delta;  // kInf: no buckets
    int32_t mode;
    uint32_t dense_thresh;
    int32_t small_max;
    int32_t chunk_edges;
    int32_t cfg;
    long long deadline_ns;
};

struct SweepCtx {
    uint32_t k;                    // current sweep
    unsigned long long bucket_hi;  // exclusive bound of the current bucket
    uint32_t fa;                   // far-list generation
    bool dense_next;               // small advances are only stamped
    unsigned long long items = 0, edges = 0, adv = 0;
    uint32_t stamped = 0;          // small vertices stamped for the next sweep (dense_next)
};

__device__ __forceinline__ uint32_t stamp_word(uint32_t sweep, uint32_t cls) { return (sweep << 2) | cls; }

// Put v (already advanced) into the worklist of sweep k+1.  Warp-collective.
template <typename OffT>
__device__ __forceinline__ void push_near(const GraphArgs<OffT> &a, bool want, int32_t v, SweepCtx &c) {
    const uint32_t nk = c.k + 1;
    bool newly = false;
    uint32_t cls = 0;
    if (want) {
        const uint32_t s = __ldcg(a.stamp + v);
        cls = s & 3u;
        if (cls != 0 && (s >> 2) < nk) {
            if (c.dense_next && cls == 1) {
                atomicMax(a.stamp + v, stamp_word(nk, 1));  // result unused: a reduction
                c.stamped++;
            } else {
                newly = (atomicMax(a.stamp + v, stamp_word(nk, cls)) >> 2) < nk;
            }
        }
    }
    const uint32_t nx = nk % 3;
    const bool is_small = newly && cls == 1;
    const bool is_large = newly && cls == 2;
    if (__any_sync(0xffffffffu, is_small)) {
        const uint32_t slot = warp_append_slot(is_small, &a.h->n_small[nx]);
        if (is_small) a.small[nk & 1][slot] = v;
    }
    if (__any_sync(0xffffffffu, is_large)) {
        uint32_t nch = 0;
        if (is_large) {
            const uint32_t deg = (uint32_t)(__ldg(a.off + v + 1) - __ldg(a.off + v));
            nch = (deg + a.chunk_edges - 1) / a.chunk_edges;
        }
        const uint32_t base = warp_reserve(nch, &a.h->n_chunk[nx]);
        int2 *dst = a.chunk[nk & 1] + base;
        for (uint32_t q = 0; q < nch; q++) dst[q] = make_int2(v, (int)q);
    }
}

// Evaluate forbidden(v) against candidate distances and advance, for up to
// kUnroll arcs per lane.  Warp-collective.
template <typename OffT>
__device__ __forceinline__ void relax_multi(const GraphArgs<OffT> &a, const bool (&ok)[kUnroll],
                                            const int32_t (&v)[kUnroll], const uint64_t (&cand64)[kUnroll],
                                            SweepCtx &c) {
    uint32_t dv[kUnroll];
#pragma unroll
    for (int j = 0; j < kUnroll; j++) dv[j] = ok[j] ? __ldcg(a.dist + v[j]) : 0u;
    bool improved[kUnroll];
#pragma unroll
    for (int j = 0; j < kUnroll; j++) {
        improved[j] = false;
        if (ok[j]) {
            if (cand64[j] >= (uint64_t)kInf) {
                set_status(a.h, LLP_ERR_OVERFLOW);
            } else if ((uint32_t)cand64[j] < dv[j]) {
                improved[j] = (uint32_t)cand64[j] < atomicMin(a.dist + v[j], (uint32_t)cand64[j]);
            }
        }
        c.adv += improved[j];
    }
#pragma unroll
    for (int j = 0; j < kUnroll; j++) {
        if (!__any_sync(0xffffffffu, improved[j])) continue;
        const uint32_t cand = (uint32_t)cand64[j];
        bool near = improved[j] && (unsigned long long)cand < c.bucket_hi;
        const bool far = improved[j] && !near;
        if (__any_sync(0xffffffffu, far)) {
            const uint32_t slot = warp_append_slot(far, &a.h->n_far[c.fa % 3]);
            if (far) {
                if (slot < a.far_cap) {
                    a.far[c.fa & 1][slot] = make_int2(v[j], (int)cand);
                    atomicMin(&a.h->far_min[c.fa % 3], cand);
                } else {
                    near = true;  // far list full: keep it in the near worklist (still correct)
                }
            }
        }
        push_near(a, near, v[j], c);
    }
}

// Expand the out-arcs of up to 32 small vertices (one per lane) edge-balanced
// across the warp, kUnroll batches of 32 arcs at a time.
template <typename OffT, bool UNIT>
__device__ __forceinline__ void expand_group(const GraphArgs<OffT> &a, bool valid, int32_t u, SweepCtx &c) {
    uint32_t du = 0, deg = 0;
    OffT beg = 0;
    if (valid) {
        du = __ldcg(a.dist + u);
        beg = __ldg(a.off + u);
        deg = (uint32_t)(__ldg(a.off + u + 1) - beg);
    }
    c.items += valid;
    uint32_t incl = deg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane_id() >= o) incl += t;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t excl = incl - deg;
    c.edges += (lane_id() == 0) ? total : 0;
    for (uint32_t base = 0; base < total; base += 32 * kUnroll) {
        bool ok[kUnroll];
        int32_t v[kUnroll];
        uint64_t cand[kUnroll];
#pragma unroll
        for (int j = 0; j < kUnroll; j++) {
            const uint32_t t = base + 32 * j + lane_id();
            int pos = 0;
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) {
                const uint32_t probe = __shfl_sync(0xffffffffu, incl, pos + s - 1);
                if (probe <= t) pos += s;
            }
            ok[j] = t < total;
            const int owner = ok[j] ? pos : 0;
            const uint32_t ex = __shfl_sync(0xffffffffu, excl, owner);
            const OffT bo = __shfl_sync(0xffffffffu, beg, owner);
            const uint32_t dq = __shfl_sync(0xffffffffu, du, owner);
            v[j] = 0;
            uint32_t w = 0;
            if (ok[j]) {
                const OffT e = bo + (OffT)(t - ex);
                v[j] = __ldg(a.idx + e);
                w = UNIT ? 1u : __ldg(a.w + e);
            }
            cand[j] = (uint64_t)dq + w;
        }
        relax_multi(a, ok, v, cand, c);
    }
}

// One chunk (<= chunk_edges arcs) of one large vertex.
template <typename OffT, bool UNIT>
__device__ __forceinline__ void expand_chunk(const GraphArgs<OffT> &a, int2 item, SweepCtx &c) {
    const int32_t u = item.x;
    uint32_t su = 0, du = 0;
    if (lane_id() == 0) {
        su = __ldcg(a.stamp + u);
        du = __ldcg(a.dist + u);
    }
    su = __shfl_sync(0xffffffffu, su, 0);
    du = __shfl_sync(0xffffffffu, du, 0);
    if ((su >> 2) != c.k) return;  // re-advanced meanwhile: sweep k+1 handles it (warp-uniform)
    const OffT b0 = __ldg(a.off + u);
    const OffT e0 = __ldg(a.off + u + 1);
    const OffT beg = b0 + (OffT)item.y * (OffT)a.chunk_edges;
    const OffT end = min(e0, beg + (OffT)a.chunk_edges);
    c.items += (lane_id() == 0 && item.y == 0);
    c.edges += (lane_id() == 0) ? (unsigned long long)(end - beg) : 0ull;
    for (OffT base = beg; base < end; base += 32 * kUnroll) {
        bool ok[kUnroll];
        int32_t v[kUnroll];
        uint64_t cand[kUnroll];
#pragma unroll
        for (int j = 0; j < kUnroll; j++) {
            const OffT e = base + 32 * j + lane_id();
            ok[j] = e < end;
            v[j] = 0;
            uint32_t w = 0;
            if (ok[j]) {
                v[j] = __ldg(a.idx + e);
                w = UNIT ? 1u : __ldg(a.w + e);
            }
            cand[j] = (uint64_t)du + w;
        }
        relax_multi(a, ok, v, cand, c);
    }
}

// Adds the CTA's dense_next stamp count to the next sweep's counter.
__device__ __forceinline__ void flush_stamped(WsHeader *h, SweepCtx &c, uint32_t *s_cnt) {
    const uint32_t ws = warp_sum(c.stamped);
    c.stamped = 0;
    if (lane_id() == 0 && ws) atomicAdd(s_cnt, ws);
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t t = *s_cnt;
        *s_cnt = 0;
        if (t) atomicAdd(&h->n_small[(c.k + 1) % 3], t);
    }
}

template <typename OffT, bool UNIT>
__global__ void __launch_bounds__(512, 2) graph_sweep_kernel(GraphArgs<OffT> a) {
    __shared__ uint32_t s_cnt;
    WsHeader *h = a.h;
    const long long t0 = globaltimer_ns();
    const long long deadline = t0 + a.deadline_ns;
    uint32_t phase = 0;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
    const int warps_per_block = blockDim.x >> 5;
    const int64_t gwarp = (int64_t)blockIdx.x * warps_per_block + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * warps_per_block;
    if (threadIdx.x == 0) s_cnt = 0;

    // ---- init_global_state / initial_states_to_process (paper Sec. 3.3)
    for (int64_t v = gtid; v < a.n; v += gthreads) {
        const uint32_t deg = (uint32_t)(__ldg(a.off + v + 1) - __ldg(a.off + v));
        const uint32_t cls = deg == 0 ? 0u : (deg <= (uint32_t)a.small_max ? 1u : 2u);
        a.dist[v] = (v == a.source) ? 0u : kInf;
        a.stamp[v] = stamp_word((v == a.source && cls) ? 1u : 0u, cls);
    }
    if (gtid == 0) {
        h->t_start = t0;
        h->mode_used = a.mode;
        h->delta_used = a.delta;
        h->block_cfg_used = a.cfg;
        for (int i = 0; i < 3; i++) h->far_min[i] = kInf;
        h->list_ok[1] = 1;
        const uint32_t src_deg = (uint32_t)(__ldg(a.off + a.source + 1) - __ldg(a.off + a.source));
        if (src_deg > 0) {
            if (src_deg <= (uint32_t)a.small_max) {
                a.small[1][0] = a.source;
                h->n_small[1] = 1;
            } else {
                const uint32_t nch = (src_deg + a.chunk_edges - 1) / a.chunk_edges;
                for (uint32_t q = 0; q < nch; q++) a.chunk[1][q] = make_int2(a.source, (int)q);
                h->n_chunk[1] = nch;
            }
        }
    }
    bool alive = grid_barrier(h, phase, deadline);

    SweepCtx c;
    c.k = 1;
    c.fa = 0;
    c.bucket_hi = (a.delta == kInf) ? (1ull << 40) : (unsigned long long)a.delta;
    uint32_t dense_sweeps = 0;
    while (alive) {
        const uint32_t k = c.k;
        const uint32_t ns = *(volatile uint32_t *)&h->n_small[k % 3];
        const uint32_t nc = *(volatile uint32_t *)&h->n_chunk[k % 3];
        const bool list_ok = *(volatile uint32_t *)&h->list_ok[k % 3] != 0;
        const bool dense = ns + nc > 0 &&
                           (!list_ok || a.mode == LLP_MODE_DENSE || (a.mode == LLP_MODE_AUTO && ns > a.dense_thresh));
        c.dense_next = dense && a.mode != LLP_MODE_SPARSE;
        if (gtid == 0) {
            const uint32_t r = (k + 2) % 3;
            h->n_small[r] = 0;
            h->n_chunk[r] = 0;
            h->list_ok[r] = 0;
            h->list_ok[(k + 1) % 3] = c.dense_next ? 0u : 1u;
            if (k - 1 < kSweepLogCap)
                sweep_log(h)[k - 1] = SweepRec{(uint32_t)(globaltimer_ns() - t0), ns, nc,
                                               (dense ? 1u : 0u) | (ns + nc == 0 ? 2u : 0u)};
        }
        if (ns + nc == 0) {
            // near worklist empty: move to the next non-empty bucket, or stop
            const uint32_t nf_raw = *(volatile uint32_t *)&h->n_far[c.fa % 3];
            const uint32_t nf = min(nf_raw, a.far_cap);
            if (nf == 0) break;
            c.dense_next = false;
            const unsigned long long fmin = *(volatile uint32_t *)&h->far_min[c.fa % 3];
            const unsigned long long dl = a.delta;
            unsigned long long nh = (fmin / dl + 1ull) * dl;
            if (nh < c.bucket_hi + dl) nh = c.bucket_hi + dl;
            if (gtid == 0) {
                h->n_far[(c.fa + 2) % 3] = 0;
                h->far_min[(c.fa + 2) % 3] = kInf;
                h->list_ok[(k + 1) % 3] = 1;
                h->aux += 1;
            }
            const int2 *fl = a.far[c.fa & 1];
            for (int64_t base = gwarp * 32; base < nf; base += nwarps * 32) {
                const int64_t i = base + lane_id();
                const bool ok = i < nf;
                int2 e = make_int2(0, 0);
                bool live = false;
                if (ok) {
                    e = fl[i];
                    live = __ldcg(a.dist + e.x) == (uint32_t)e.y;
                }
                bool to_near = live && (unsigned long long)(uint32_t)e.y < nh;
                const bool keep = live && !to_near;
                const uint32_t slot = warp_append_slot(keep, &h->n_far[(c.fa + 1) % 3]);
                if (keep) {
                    if (slot < a.far_cap) {
                        a.far[(c.fa + 1) & 1][slot] = e;
                        atomicMin(&h->far_min[(c.fa + 1) % 3], (uint32_t)e.y);
                    } else {
                        to_near = true;
                    }
                }
                push_near(a, to_near, e.x, c);
            }
            c.bucket_hi = nh;
            c.fa += 1;
        } else {
            dense_sweeps += dense;
            const uint32_t ngroups =
                dense ? (uint32_t)(((int64_t)a.n + 31) / 32) : (uint32_t)(((uint64_t)ns + 31) / 32);
            const int2 *cl = a.chunk[k & 1];
            const int32_t *sl = a.small[k & 1];
            const int64_t total = (int64_t)nc + ngroups;
            for (int64_t it = gwarp; it < total; it += nwarps) {
                if (it < nc) {
                    expand_chunk<OffT, UNIT>(a, cl[it], c);
                } else {
                    const int64_t g = it - nc;
                    int32_t u = 0;
                    bool ok;
                    if (dense) {
                        const int64_t vv = g * 32 + lane_id();
                        ok = vv < a.n;
                        u = ok ? (int32_t)vv : 0;
                        if (ok) ok = __ldcg(a.stamp + u) == stamp_word(k, 1);
                    } else {
                        const int64_t i = g * 32 + lane_id();
                        ok = i < ns;
                        u = ok ? sl[i] : 0;
                        if (ok) ok = (__ldcg(a.stamp + u) >> 2) == k;
                    }
                    expand_group<OffT, UNIT>(a, ok, u, c);
                }
            }
        }
        flush_stamped(h, c, &s_cnt);
        alive = grid_barrier(h, phase, deadline);
        c.k += 1;
    }

    // ---- statistics (one atomic per warp)
    const unsigned long long it_s = warp_sum(c.items), ed_s = warp_sum(c.edges), ad_s = warp_sum(c.adv);
    if (lane_id() == 0) {
        atomicAdd(&h->items, it_s);
        atomicAdd(&h->edges, ed_s);
        atomicAdd(&h->advances, ad_s);
    }
    if (gtid == 0) {
        h->sweeps = (int32_t)c.k;
        h->dense_sweeps = (int32_t)dense_sweeps;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t done = atomicAdd(&h->scratch[0], 1u) + 1u;
        if (done == gridDim.x) h->t_end = globaltimer_ns();
    }
}

struct Layout {
    uint32_t *stamp;
    int32_t *small[2];
    int2 *chunk[2];
    int2 *far[2];
    uint32_t far_cap;
    size_t bytes;
};

Layout carve_graph(void *ws, int32_t n, int64_t m) {
    Carve c(ws);
    Layout L;
    // chunks of one sweep: sum over large v of ceil(deg/chunk) <= m/128 + m/17
    const size_t chunk_cap = (size_t)(m / 128 + m / 16 + 2);
    L.far_cap = (uint32_t)std::max<int64_t>(n, 1024);
    L.stamp = c.take<uint32_t>(n);
    L.small[0] = c.take<int32_t>(n);
    L.small[1] = c.take<int32_t>(n);
    L.chunk[0] = c.take<int2>(chunk_cap);
    L.chunk[1] = c.take<int2>(chunk_cap);
    L.far[0] = c.take<int2>(L.far_cap);
    L.far[1] = c.take<int2>(L.far_cap);
    L.bytes = c.bytes();
    return L;
}

// Heuristic schedule (the fallback of the learned scheduler).
void resolve_schedule(const llp_sched_t *s, bool unit, int32_t n, int64_t m, int32_t &mode, uint32_t &delta,
                      int32_t &cfg, uint32_t &dense_thresh, int &threads) {
    mode = s ? s->mode : LLP_MODE_AUTO;
    if (mode < 0 || mode > 2) mode = LLP_MODE_AUTO;
    delta = s ? s->delta : 0u;
    if (delta == 0u) delta = kInf;  // heuristic: one worklist
    if (unit) delta = kInf;         // unit weights: sweeps are BFS levels already
    cfg = s ? s->block_cfg : 0;
    if (cfg < 1 || cfg > LLP_BLOCK_CFGS) cfg = 2;
    const int pm = (s && s->dense_permille > 0) ? s->dense_permille : 50;
    dense_thresh = (uint32_t)std::min<int64_t>((int64_t)n * pm / 1000, 0xFFFFFFFFll);
    threads = (s && (s->threads == 256 || s->threads == 512)) ? s->threads : 512;
    (void)m;
}

template <bool UNIT>
llp_status_t graph_solve(const llp_csr_t *g, int32_t source, uint32_t *out, const llp_sched_t *s, void *ws,
                         size_t ws_bytes, cudaStream_t stream) {
    if (!g || !out || !ws) return LLP_ERR_INVALID_ARG;
    if (g->n < 1 || g->n > (1 << 29) || g->m < 0 || !g->offsets) return LLP_ERR_INVALID_ARG;
    if (g->m > 0 && (!g->indices || (!UNIT && !g->weights))) return LLP_ERR_INVALID_ARG;
    if (!g->offsets_64 && g->m > 0x7FFFFFFFll) return LLP_ERR_INVALID_ARG;
    if (source < 0 || source >= g->n) return LLP_ERR_INVALID_ARG;
    if (((uintptr_t)ws & 255u) != 0) return LLP_ERR_INVALID_ARG;
    Layout L = carve_graph(ws, g->n, g->m);
    if (ws_bytes < L.bytes) return LLP_ERR_WORKSPACE_TOO_SMALL;

    int32_t mode, cfg;
    uint32_t delta, dense_thresh;
    int threads;
    resolve_schedule(s, UNIT, g->n, g->m, mode, delta, cfg, dense_thresh, threads);
    const BlockCfg bc = block_cfg_of(cfg);
    llp_status_t rc = reset_header(ws, stream);
    if (rc != LLP_OK) return rc;

    auto fill = [&](auto &args) {
        args.n = g->n;
        args.source = source;
        args.idx = g->indices;
        args.w = UNIT ? nullptr : g->weights;
        args.dist = out;
        args.stamp = L.stamp;
        args.small[0] = L.small[0];
        args.small[1] = L.small[1];
        args.chunk[0] = L.chunk[0];
        args.chunk[1] = L.chunk[1];
        args.far[0] = L.far[0];
        args.far[1] = L.far[1];
        args.far_cap = L.far_cap;
        args.h = (WsHeader *)ws;
        args.delta = delta;
        args.mode = mode;
        args.dense_thresh = dense_thresh;
        args.small_max = bc.small_max;
        args.chunk_edges = bc.chunk;
        args.cfg = cfg;
        args.deadline_ns = deadline_from(s);
    };
    if (g->offsets_64) {
        GraphArgs<int64_t> args;
        fill(args);
        args.off = (const int64_t *)g->offsets;
        void *kargs[] = {&args};
        return launch_cooperative((const void *)graph_sweep_kernel<int64_t, UNIT>, threads, 0, 0, kargs, stream);
    } else {
        GraphArgs<int32_t> args;
        fill(args);
        args.off = (const int32_t *)g->offsets;
        void *kargs[] = {&args};
        return launch_cooperative((const void *)graph_sweep_kernel<int32_t, UNIT>, threads, 0, 0, kargs, stream);
    }
}

}  // namespace
}  // namespace llp

extern "C" {

size_t llp_sssp_workspace_size(int32_t n, int64_t m) {
    if (n < 1 || m < 0) return 0;
    return llp::carve_graph(nullptr, n, m).bytes;
}

size_t llp_bfs_workspace_size(int32_t n, int64_t m) { return llp_sssp_workspace_size(n, m); }

llp_status_t llp_sssp(const llp_csr_t *g, int32_t source, uint32_t *dist, const llp_sched_t *sched, void *ws,
                      size_t ws_bytes, void *stream) {
    return llp::graph_solve<false>(g, source, dist, sched, ws, ws_bytes, (cudaStream_t)stream);
}

llp_status_t llp_bfs(const llp_csr_t *g, int32_t source, uint32_t *level, const llp_sched_t *sched, void *ws,
                     size_t ws_bytes, void *stream) {
    return llp::graph_solve<true>(g, source, level, sched, ws, ws_bytes, (cudaStream_t)stream);
}

}  // extern "C"

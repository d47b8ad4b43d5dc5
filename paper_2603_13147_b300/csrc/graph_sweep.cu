// Persistent forbidden/advance sweep engine for the graph problems:
// SSSP (paper Sec. 4.1) and BFS (paper Sec. 4.2).
//
// State G = dist[] (uint32, 0xFFFFFFFF = "infinity").  A vertex v is forbidden
// when some arc (u, v) offers d(u) + w(u, v) < d(v); the advance lowers d(v)
// with atomicMin, which is the lock-free monotone update the paper's
// requirements list (Sec. 3.2: atomic, monotone, progress detection).  The
// predicate is evaluated push-style: when u is taken from the worklist, each of
// its out-arcs is checked, and every successful advance puts v into the next
// worklist (the paper's problem-specific state selection, Sec. 3.2).
//
// One cooperative launch runs all sweeps; sweeps are separated by a bounded
// grid barrier.  Per sweep k:
//   - worklist items are (a) "small" vertices (out-degree <= small_max), taken
//     32 per warp and expanded edge-balanced inside the warp, and (b) chunks of
//     <= chunk arcs of the larger vertices, one chunk per warp, so hubs are
//     spread over the whole grid;
//   - sparse mode walks the small-vertex list; dense mode instead scans every
//     vertex's stamp (the paper's all-indices solver) and touches the CSR in
//     vertex order;
//   - stamp[v] == k marks "v is in the worklist of sweep k"; atomicMax on the
//     stamp deduplicates appends, appends are warp-aggregated (ballot/popc);
//   - with a finite bucket width delta (the paper's bucket worklist, Sec. 3.3
//     "parallel buckets"), only advances with d < current bucket bound enter
//     the next worklist; the others wait in a far list that is filtered when
//     the near worklist empties.
// The sweep stops when no index is forbidden: both worklists are empty.
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

struct LocalStats {
    unsigned long long items = 0, edges = 0, adv = 0;
};

// Put v (already advanced) into the worklist of sweep k+1.  Warp-collective.
template <typename OffT>
__device__ __forceinline__ void push_near(const GraphArgs<OffT> &a, bool want, int32_t v, uint32_t k) {
    uint32_t deg = 0;
    bool newly = false;
    if (want) {
        const OffT b = __ldg(a.off + v);
        const OffT e = __ldg(a.off + v + 1);
        deg = (uint32_t)(e - b);
        if (deg > 0) newly = atomicMax(a.stamp + v, k + 1) < k + 1;
    }
    const uint32_t nx = (k + 1) % 3;
    const bool is_small = newly && deg <= (uint32_t)a.small_max;
    const bool is_large = newly && deg > (uint32_t)a.small_max;
    const uint32_t slot = warp_append_slot(is_small, &a.h->n_small[nx]);
    if (is_small) a.small[(k + 1) & 1][slot] = v;
    const uint32_t nch = is_large ? (deg + a.chunk_edges - 1) / a.chunk_edges : 0u;
    const uint32_t base = warp_reserve(nch, &a.h->n_chunk[nx]);
    int2 *dst = a.chunk[(k + 1) & 1] + base;
    for (uint32_t c = 0; c < nch; c++) dst[c] = make_int2(v, (int)c);
}

// Evaluate forbidden(v) against one candidate and advance.  Warp-collective:
// all 32 lanes call it; `valid` masks lanes without an arc.
template <typename OffT>
__device__ __forceinline__ void relax(const GraphArgs<OffT> &a, bool valid, int32_t v, uint64_t cand64, uint32_t k,
                                      unsigned long long bucket_hi, uint32_t fa, LocalStats &st) {
    bool improved = false;
    uint32_t cand = 0;
    if (valid) {
        if (cand64 >= (uint64_t)kInf) {
            set_status(a.h, LLP_ERR_OVERFLOW);
        } else {
            cand = (uint32_t)cand64;
            const uint32_t dv = __ldcg(a.dist + v);
            if (cand < dv) {
                const uint32_t old = atomicMin(a.dist + v, cand);
                improved = cand < old;
            }
        }
    }
    st.adv += improved;
    bool near = improved && (unsigned long long)cand < bucket_hi;
    const bool far = improved && !near;
    if (__any_sync(0xffffffffu, far)) {
        const uint32_t slot = warp_append_slot(far, &a.h->n_far[fa % 3]);
        if (far) {
            if (slot < a.far_cap) {
                a.far[fa & 1][slot] = make_int2(v, (int)cand);
                atomicMin(&a.h->far_min[fa % 3], cand);
            } else {
                near = true;  // far list full: keep it in the near worklist (still correct)
            }
        }
    }
    if (__any_sync(0xffffffffu, near)) push_near(a, near, v, k);
}

// Expand the out-arcs of up to 32 small vertices (one per lane) edge-balanced
// across the warp.
template <typename OffT, bool UNIT>
__device__ __forceinline__ void expand_group(const GraphArgs<OffT> &a, bool valid, int32_t u, uint32_t k,
                                             unsigned long long bucket_hi, uint32_t fa, LocalStats &st) {
    uint32_t du = 0, deg = 0;
    OffT beg = 0;
    if (valid) {
        du = __ldcg(a.dist + u);
        beg = __ldg(a.off + u);
        deg = (uint32_t)(__ldg(a.off + u + 1) - beg);
    }
    st.items += valid;
    uint32_t incl = deg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane_id() >= o) incl += t;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t excl = incl - deg;
    st.edges += (lane_id() == 0) ? total : 0;
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t t = base + lane_id();
        int pos = 0;
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
            const uint32_t probe = __shfl_sync(0xffffffffu, incl, pos + s - 1);
            if (probe <= t) pos += s;
        }
        const bool ok = t < total;
        const int owner = ok ? pos : 0;
        const uint32_t ex = __shfl_sync(0xffffffffu, excl, owner);
        const OffT bo = __shfl_sync(0xffffffffu, beg, owner);
        const uint32_t dq = __shfl_sync(0xffffffffu, du, owner);
        int32_t v = 0;
        uint32_t w = 0;
        if (ok) {
            const OffT e = bo + (OffT)(t - ex);
            v = __ldg(a.idx + e);
            w = UNIT ? 1u : __ldg(a.w + e);
        }
        relax(a, ok, v, (uint64_t)dq + w, k, bucket_hi, fa, st);
    }
}

// One chunk (<= chunk_edges arcs) of one large vertex.
template <typename OffT, bool UNIT>
__device__ __forceinline__ void expand_chunk(const GraphArgs<OffT> &a, int2 item, uint32_t k,
                                             unsigned long long bucket_hi, uint32_t fa, LocalStats &st) {
    const int32_t u = item.x;
    uint32_t su = 0, du = 0;
    if (lane_id() == 0) {
        su = __ldcg(a.stamp + u);
        du = __ldcg(a.dist + u);
    }
    su = __shfl_sync(0xffffffffu, su, 0);
    du = __shfl_sync(0xffffffffu, du, 0);
    if (su != k) return;  // re-advanced meanwhile: sweep k+1 handles it (warp-uniform)
    const OffT b0 = __ldg(a.off + u);
    const OffT e0 = __ldg(a.off + u + 1);
    const OffT beg = b0 + (OffT)item.y * (OffT)a.chunk_edges;
    const OffT end = min(e0, beg + (OffT)a.chunk_edges);
    st.items += (lane_id() == 0 && item.y == 0);
    st.edges += (lane_id() == 0) ? (unsigned long long)(end - beg) : 0ull;
    for (OffT base = beg; base < end; base += 32) {
        const OffT e = base + lane_id();
        const bool ok = e < end;
        int32_t v = 0;
        uint32_t w = 0;
        if (ok) {
            v = __ldg(a.idx + e);
            w = UNIT ? 1u : __ldg(a.w + e);
        }
        relax(a, ok, v, (uint64_t)du + w, k, bucket_hi, fa, st);
    }
}

template <typename OffT, bool UNIT>
__global__ void __launch_bounds__(512) graph_sweep_kernel(GraphArgs<OffT> a) {
    WsHeader *h = a.h;
    const long long t0 = globaltimer_ns();
    const long long deadline = t0 + a.deadline_ns;
    uint32_t phase = 0;
    LocalStats st;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
    const int warps_per_block = blockDim.x >> 5;
    const int64_t gwarp = (int64_t)blockIdx.x * warps_per_block + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * warps_per_block;

    // ---- init_global_state / initial_states_to_process (paper Sec. 3.3)
    const uint32_t src_deg = (uint32_t)(__ldg(a.off + a.source + 1) - __ldg(a.off + a.source));
    for (int64_t v = gtid; v < a.n; v += gthreads) {
        a.dist[v] = (v == a.source) ? 0u : kInf;
        a.stamp[v] = (v == a.source && src_deg > 0) ? 1u : 0u;
    }
    if (gtid == 0) {
        h->t_start = t0;
        h->mode_used = a.mode;
        h->delta_used = a.delta;
        h->block_cfg_used = a.cfg;
        for (int i = 0; i < 3; i++) h->far_min[i] = kInf;
        if (src_deg > 0) {
            if (src_deg <= (uint32_t)a.small_max) {
                a.small[1][0] = a.source;
                h->n_small[1] = 1;
            } else {
                const uint32_t nch = (src_deg + a.chunk_edges - 1) / a.chunk_edges;
                for (uint32_t c = 0; c < nch; c++) a.chunk[1][c] = make_int2(a.source, (int)c);
                h->n_chunk[1] = nch;
            }
        }
    }
    bool alive = grid_barrier(h, phase, deadline);

    uint32_t k = 1, fa = 0, dense_sweeps = 0;
    unsigned long long bucket_hi = (a.delta == kInf) ? (1ull << 40) : (unsigned long long)a.delta;
    while (alive) {
        const uint32_t ns = *(volatile uint32_t *)&h->n_small[k % 3];
        const uint32_t nc = *(volatile uint32_t *)&h->n_chunk[k % 3];
        if (gtid == 0) {
            const uint32_t r = (k + 2) % 3;
            h->n_small[r] = 0;
            h->n_chunk[r] = 0;
        }
        if (ns + nc == 0) {
            // near worklist empty: move to the next non-empty bucket, or stop
            const uint32_t nf_raw = *(volatile uint32_t *)&h->n_far[fa % 3];
            const uint32_t nf = min(nf_raw, a.far_cap);
            if (nf == 0) break;
            const unsigned long long fmin = *(volatile uint32_t *)&h->far_min[fa % 3];
            const unsigned long long dl = a.delta;
            unsigned long long nh = (fmin / dl + 1ull) * dl;
            if (nh < bucket_hi + dl) nh = bucket_hi + dl;
            if (gtid == 0) {
                h->n_far[(fa + 2) % 3] = 0;
                h->far_min[(fa + 2) % 3] = kInf;
                h->aux += 1;
            }
            const int2 *fl = a.far[fa & 1];
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
                const uint32_t slot = warp_append_slot(keep, &h->n_far[(fa + 1) % 3]);
                if (keep) {
                    if (slot < a.far_cap) {
                        a.far[(fa + 1) & 1][slot] = e;
                        atomicMin(&h->far_min[(fa + 1) % 3], (uint32_t)e.y);
                    } else {
                        to_near = true;
                    }
                }
                push_near(a, to_near, e.x, k);
            }
            bucket_hi = nh;
            fa += 1;
        } else {
            const bool dense = a.mode == LLP_MODE_DENSE || (a.mode == LLP_MODE_AUTO && ns > a.dense_thresh);
            dense_sweeps += dense;
            const uint32_t ngroups = dense ? (uint32_t)(((int64_t)a.n + 31) / 32) : (uint32_t)(((uint64_t)ns + 31) / 32);
            const int2 *cl = a.chunk[k & 1];
            const int32_t *sl = a.small[k & 1];
            const int64_t total = (int64_t)nc + ngroups;
            for (int64_t it = gwarp; it < total; it += nwarps) {
                if (it < nc) {
                    expand_chunk<OffT, UNIT>(a, cl[it], k, bucket_hi, fa, st);
                } else {
                    const int64_t g = it - nc;
                    int32_t u = 0;
                    bool ok;
                    if (dense) {
                        const int64_t vv = g * 32 + lane_id();
                        ok = vv < a.n;
                        u = ok ? (int32_t)vv : 0;
                        if (ok) ok = __ldcg(a.stamp + u) == k;
                        if (ok) ok = (__ldg(a.off + u + 1) - __ldg(a.off + u)) <= (OffT)a.small_max;
                    } else {
                        const int64_t i = g * 32 + lane_id();
                        ok = i < ns;
                        u = ok ? sl[i] : 0;
                        if (ok) ok = __ldcg(a.stamp + u) == k;
                    }
                    expand_group<OffT, UNIT>(a, ok, u, k, bucket_hi, fa, st);
                }
            }
        }
        alive = grid_barrier(h, phase, deadline);
        k += 1;
    }

    // ---- statistics (one atomic per warp)
    const unsigned long long it_s = warp_sum(st.items), ed_s = warp_sum(st.edges), ad_s = warp_sum(st.adv);
    if (lane_id() == 0) {
        atomicAdd(&h->items, it_s);
        atomicAdd(&h->edges, ed_s);
        atomicAdd(&h->advances, ad_s);
    }
    if (gtid == 0) {
        h->sweeps = (int32_t)k;
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
    if (g->n < 1 || g->m < 0 || !g->offsets) return LLP_ERR_INVALID_ARG;
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

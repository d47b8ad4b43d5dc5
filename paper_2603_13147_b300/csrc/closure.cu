// Transitive closure as an LLP (paper Sec. 4.6), bit-packed.
//
// G[u,v] is bit (v & 31) of word reach[u*W + v/32], W = ceil(n/32).  The pair
// (u,v) is forbidden when G[u,v] is 0 but G[u,w] and G[w,v] are 1 for some w;
// it suffices to take w among u's direct successors (any path's first arc), so
// the advance of row u is  G[u] |= G[w]  for the successors w.  Sweep 1 uses
// every successor; sweep k > 1 only the successors whose row gained bits in
// sweep k-1 (their earlier bits are already in G[u]).  One warp owns a row
// during a sweep and writes it with plain stores; other warps read it
// concurrently, which is safe because rows only gain bits (monotone).  popc
// counts the pairs each advance adds.  Stops after a sweep that adds nothing.
#include "llp_common.cuh"

#ifndef LLP_READ_ONCE
#define LLP_READ_ONCE 1
#endif

namespace llp {
namespace {

constexpr int kClosureSlices = 8;  // row words per lane per pass (256 words = 8,192 columns)

template <typename OffT>
struct ClosureArgs {
    int32_t n;
    int32_t W;
    const OffT *off;
    const int32_t *idx;
    uint32_t *reach;
    uint8_t *changed[3];
    WsHeader *h;
    long long deadline_ns;
};

template <typename OffT>
__global__ void __launch_bounds__(512) closure_kernel(ClosureArgs<OffT> a) {
    WsHeader *h = a.h;
    const long long t0 = globaltimer_ns();
    const long long deadline = t0 + a.deadline_ns;
    uint32_t phase = 0;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
    const int wpb = blockDim.x >> 5;
    const int64_t gwarp = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * wpb;
    const int64_t words = (int64_t)a.n * a.W;
    const int64_t m = (int64_t)__ldg(a.off + a.n);
    unsigned long long rows_adv = 0, ors = 0, bits = 0;
    __shared__ uint32_t s_any;

    // init_global_state: G = adjacency
    for (int64_t x = gtid; x < words; x += gthreads) a.reach[x] = 0u;
    for (int64_t u = gtid; u < a.n; u += gthreads) {
        a.changed[0][u] = 0;
        a.changed[1][u] = 0;
        a.changed[2][u] = 0;
    }
    if (gtid == 0) h->t_start = t0;
    bool alive = grid_barrier(h, phase, deadline);
    if (alive) {
        // arc (u, v): set bit v of row u; u is found by the warp walking rows
        for (int64_t u = gwarp; u < a.n; u += nwarps) {
            const OffT b = __ldg(a.off + u), e = __ldg(a.off + u + 1);
            for (OffT x = b + lane_id(); x < e; x += 32) {
                const int32_t v = __ldg(a.idx + x);
                atomicOr(a.reach + u * (int64_t)a.W + (v >> 5), 1u << (v & 31));
            }
        }
        alive = grid_barrier(h, phase, deadline);
    }
    uint32_t k = 1;
    while (alive) {
        if (threadIdx.x == 0) s_any = 0;
        __syncthreads();
        const uint8_t *prev = a.changed[(k + 2) % 3];
        uint8_t *cur = a.changed[k % 3];
        uint8_t *clear = a.changed[(k + 1) % 3];
        for (int64_t u = gtid; u < a.n; u += gthreads) clear[u] = 0;
        for (int64_t u = gwarp; u < a.n; u += nwarps) {
            const OffT b = __ldg(a.off + u), e = __ldg(a.off + u + 1);
            if (b == e) continue;
            uint32_t *ru = a.reach + u * (int64_t)a.W;
            uint32_t gained = 0;
            // successors 32 at a time: lane j reads successor j and whether its row changed
            // in the previous sweep; then the changed rows are ORed into row u, 8 words per
            // lane (256 words) at a time, all of a successor row's loads in flight together
            for (OffT y0 = b; y0 < e; y0 += 32) {
                const OffT y = y0 + lane_id();
                const int32_t wv = y < e ? __ldg(a.idx + y) : -1;
                const bool act = wv >= 0 && (k == 1 || *(volatile const uint8_t *)(prev + wv));
                const uint32_t am = __ballot_sync(0xffffffffu, act);
                ors += (lane_id() == 0) ? (unsigned long long)__popc(am) : 0ull;
                for (int32_t c0 = 0; c0 < a.W && am; c0 += 32 * kClosureSlices) {
                    uint32_t acc[kClosureSlices];
#pragma unroll
                    for (int s = 0; s < kClosureSlices; s++) acc[s] = 0u;
                    for (uint32_t mm = am; mm; mm &= mm - 1u) {
                        const int32_t w = __shfl_sync(0xffffffffu, wv, __ffs(mm) - 1);
                        const uint32_t *rw = a.reach + w * (int64_t)a.W;
#pragma unroll
                        for (int s = 0; s < kClosureSlices; s++) {
                            const int32_t x = c0 + 32 * s + lane_id();
                            if (x < a.W) acc[s] |= __ldcg(rw + x);
                        }
                    }
#pragma unroll
                    for (int s = 0; s < kClosureSlices; s++) {
                        const int32_t x = c0 + 32 * s + lane_id();
                        if (x < a.W) {
                            const uint32_t old = ru[x];
                            const uint32_t add = acc[s] & ~old;
                            if (add) {
                                ru[x] = old | add;
                                gained += __popc(add);
                            }
                        }
                    }
                }
            }
            const uint32_t g = warp_sum(gained);
            if (g) {
                if (lane_id() == 0) {
                    cur[u] = 1;
                    s_any = 1;
                }
                bits += (lane_id() == 0) ? g : 0;
                rows_adv += (lane_id() == 0);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && s_any) atomicOr(&h->scratch[1 + (k & 1)], 1u);
        if (gtid == 0) h->scratch[1 + ((k + 1) & 1)] = 0;
        alive = grid_barrier(h, phase, deadline);
        if (!alive) break;
        const uint32_t any = LLP_READ_ONCE ? cta_read_once(&h->scratch[1 + (k & 1)]) : *(volatile uint32_t *)&h->scratch[1 + (k & 1)];
        k++;
        if (!any) break;
        alive = grid_barrier(h, phase, deadline);  // everyone read `any` before it is reset
    }
    const unsigned long long rs = warp_sum(rows_adv), os = warp_sum(ors), bs = warp_sum(bits);
    if (lane_id() == 0) {
        atomicAdd(&h->items, rs);
        atomicAdd(&h->edges, os);
        atomicAdd(&h->advances, bs);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t done = atomicAdd(&h->scratch[0], 1u) + 1u;
        if (done == gridDim.x) {
            h->t_end = globaltimer_ns();
            h->sweeps = (int32_t)k - 1;
        }
    }
    (void)m;
}

struct ClosureLayout {
    uint8_t *changed[3];
    size_t bytes;
};

ClosureLayout carve_closure(void *ws, int32_t n) {
    Carve c(ws);
    ClosureLayout L;
    for (int i = 0; i < 3; i++) L.changed[i] = c.take<uint8_t>(n);
    L.bytes = c.bytes();
    return L;
}

}  // namespace
}  // namespace llp

extern "C" {

size_t llp_transitive_closure_workspace_size(int32_t n, int64_t m) {
    (void)m;
    if (n < 1) return 0;
    return llp::carve_closure(nullptr, n).bytes;
}

llp_status_t llp_transitive_closure(const llp_csr_t *g, uint32_t *reach, const llp_sched_t *sched, void *ws,
                                    size_t ws_bytes, void *stream) {
    using namespace llp;
    if (!g || !reach || !ws || g->n < 1 || g->n > 65536 || g->m < 0 || !g->offsets) return LLP_ERR_INVALID_ARG;
    if (g->m > 0 && !g->indices) return LLP_ERR_INVALID_ARG;
    if (!g->offsets_64 && g->m > 0x7FFFFFFFll) return LLP_ERR_INVALID_ARG;
    if (((uintptr_t)ws & 255u) != 0) return LLP_ERR_INVALID_ARG;
    ClosureLayout L = carve_closure(ws, g->n);
    if (ws_bytes < L.bytes) return LLP_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t st = (cudaStream_t)stream;
    llp_status_t rc = reset_header(ws, st);
    if (rc != LLP_OK) return rc;
    auto fill = [&](auto &a) {
        a.n = g->n;
        a.W = (g->n + 31) / 32;
        a.idx = g->indices;
        a.reach = reach;
        for (int i = 0; i < 3; i++) a.changed[i] = L.changed[i];
        a.h = (WsHeader *)ws;
        a.deadline_ns = deadline_from(sched);
    };
    if (g->offsets_64) {
        ClosureArgs<int64_t> a;
        fill(a);
        a.off = (const int64_t *)g->offsets;
        void *args[] = {&a};
        return launch_cooperative((const void *)closure_kernel<int64_t>, 512, 0, 0, args, st);
    }
    ClosureArgs<int32_t> a;
    fill(a);
    a.off = (const int32_t *)g->offsets;
    void *args[] = {&a};
    return launch_cooperative((const void *)closure_kernel<int32_t>, 512, 0, 0, args, st);
}

}  // extern "C"

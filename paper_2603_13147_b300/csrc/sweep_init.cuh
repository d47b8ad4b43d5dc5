// init_global_state of the graph sweep (SSSP paper Sec. 4.1, BFS Sec. 4.2;
// Algorithm LLP starts from the bottom of the lattice): d = infinity except the
// source (a warm start keeps the caller's dist[]), the per-32-vertex class
// table (has out-arcs, out-degree above small_max) and cleared frontier bitmaps.
// Shared by the sweep kernel and by the learned scheduler's prologue, which
// initialises the state while other CTAs compute the schedule.
#pragma once

#include "llp_common.cuh"

namespace llp {

template <typename OffT>
struct SweepInit {
    int32_t n, source, warm;
    uint32_t small_max;
    const OffT *off;
    uint32_t *dist;
    uint2 *cls;
    uint32_t *bm0, *bm1, *bm2;
    uint32_t *fixed;  // may be NULL
};

// Warps gwarp, gwarp + nwarps, ... each take eight groups of 32 vertices per step
// (their loads in flight together).  Warp-collective.
template <typename OffT>
__device__ __forceinline__ void sweep_init(const SweepInit<OffT> &a, int64_t gwarp, int64_t nwarps) {
    for (int64_t base = gwarp * 256; base < a.n; base += nwarps * 256) {
        uint32_t deg[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const int64_t v = base + 32 * q + lane_id();
            deg[q] = v < a.n ? (uint32_t)(__ldg(a.off + v + 1) - __ldg(a.off + v)) : 0u;
        }
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const int64_t v = base + 32 * q + lane_id();
            if (v < a.n && (!a.warm || v == a.source)) a.dist[v] = (v == a.source) ? 0u : kInf;
            const uint32_t has = __ballot_sync(0xffffffffu, deg[q] > 0);
            const uint32_t large = __ballot_sync(0xffffffffu, deg[q] > a.small_max);
            if (lane_id() == 0 && base + 32 * q < a.n) {
                const int64_t wi = (base >> 5) + q;
                a.cls[wi] = make_uint2(has, large);
                if (a.fixed) a.fixed[wi] = 0u;
                a.bm0[wi] = 0u;
                a.bm1[wi] = 0u;
                a.bm2[wi] = 0u;
            }
        }
    }
}

}  // namespace llp

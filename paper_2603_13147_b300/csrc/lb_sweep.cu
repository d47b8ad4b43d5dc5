// Load-balanced forbidden/advance sweep for SSSP (paper Sec. 4.1) and BFS
// (paper Sec. 4.2) on graphs with int32 offsets and one worklist (no priority
// buckets: Bellman-Ford order, the paper's all-indices and bag solvers).
//
// Same lattice, predicate and advance as the engine in graph_sweep.cu: G[v] =
// d(v) lives in the caller's dist[]; v is forbidden when an arc (u, v) offers
// d(u) + w(u, v) < d(v); the advance is an atomic min on dist[v] (Sec. 3.2).
// What differs is how a sweep is cut into work:
//   - the worklist of sweep k is a list of entries (vertex u, first arc of u
//     in CSR, position of u's first arc in the sweep's "arc space"), the
//     positions being the running sum of the entries' out-degrees, so the arcs
//     of sweep k form one range [0, A_k);
//   - that range is cut into blocks of kBlk arcs; blk_first[b] is the entry
//     that owns arc position b * kBlk, so any warp can start on any block: the
//     work units are all the same size whatever the degrees (a hub is spread
//     over many warps, a run of tiny vertices is packed into one);
//   - a warp loads the (up to) 32 entries that cover its block, one per lane,
//     with d(u) read fresh, finds each arc's owner among them (a search over
//     the lanes' positions) and has kLbU arcs per lane in flight;
//   - an entry whose vertex was advanced again during this sweep (its bit in
//     B_{k+1} is set) is skipped: the next sweep expands it with the newer d;
//   - the next worklist is built either as a list (an advance that sets v's
//     bit in B_{k+1} first appends v, staged per warp and published with one
//     64-bit atomic add that reserves entries and arc positions together) or,
//     for wide frontiers, only as the bitmap B_{k+1} (fire-and-forget atomic
//     or), which a compaction phase after the sweep turns into the entry list.
// The run stops when a worklist holds no arc: no index is forbidden.
#include <algorithm>

#include "llp_common.cuh"

namespace llp {
namespace {

constexpr int kLbU = 8;                      // arc slots per lane per block
constexpr uint32_t kBlk = 32u * kLbU;        // arcs per block
constexpr uint32_t kLbStage = 64;            // staged appends per warp
constexpr int kLbThreads = 512;
constexpr int kLbWarps = kLbThreads / 32;
constexpr int kCompactWords = 8;             // bitmap words per lane round in the compaction

struct LbArgs {
    int32_t n, source, nwords;
    const int32_t *off;
    const int32_t *idx;
    const uint32_t *w;
    uint32_t *dist;            // state during the run, and the output
    uint32_t *bm[2];           // B_k = bm[k & 1]
    int32_t *ent_u[2];         // list k = [k & 1]
    uint32_t *ent_pos[2];
    int32_t *ent_row[2];
    uint32_t *blk_first[2];
    WsHeader *h;
    long long deadline_ns;
    unsigned long long dense_arcs;  // AUTO: the next worklist is a bitmap when this one has more arcs
    int32_t mode;
    int32_t warm, n_seeds;
    const int32_t *seeds;
};

struct LbStage {
    int32_t u[kLbStage];
    uint32_t deg[kLbStage];
    int32_t row[kLbStage];
};

__device__ __forceinline__ void red_or_u32(uint32_t *p, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.or.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_min_u32(uint32_t *p, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.min.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane_id() >= o) x += t;
    }
    return x;
}

// Number of leading lanes whose value x (non-decreasing over the lanes) is <= t,
// at most 31: with x = the lanes' inclusive prefix sums and t < the total, the
// lane that owns item t of the warp-wide concatenation.
__device__ __forceinline__ int owner_of(uint32_t incl, uint32_t t) {
    int pos = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const uint32_t probe = __shfl_sync(0xffffffffu, incl, pos + s - 1);
        if (probe <= t) pos += s;
    }
    return pos;
}

// Publishes entries (u, deg, row): reserves entries and arc positions with one
// 64-bit atomic add on the list's cursor (high word: entries, low word: arcs),
// writes them, and writes blk_first for every block whose first arc position
// falls inside one of them.  `cnt` entries, entry i given by lane i / 2's pair
// (lane l holds entries 2l and 2l+1: u0/d0/r0 and u1/d1/r1; absent ones have
// deg 0 and are never written).  Warp-collective.
__device__ __forceinline__ void publish(const LbArgs &a, uint32_t list, unsigned long long *cursor, uint32_t cnt,
                                        int32_t u0, uint32_t d0, int32_t r0, int32_t u1, uint32_t d1, int32_t r1) {
    const uint32_t loc = d0 + d1;
    const uint32_t incl = warp_incl_scan(loc);
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long base = 0;
    if (lane_id() == 31) base = atomicAdd(cursor, ((unsigned long long)cnt << 32) | total);
    base = __shfl_sync(0xffffffffu, base, 31);
    const uint32_t E0 = (uint32_t)(base >> 32);
    const uint32_t A0 = (uint32_t)base;
    const uint32_t p0 = A0 + incl - loc;
    const uint32_t p1 = p0 + d0;
    const uint32_t i0 = E0 + 2u * lane_id();
    if (2u * lane_id() < cnt) {
        a.ent_u[list][i0] = u0;
        a.ent_pos[list][i0] = p0;
        a.ent_row[list][i0] = r0;
    }
    if (2u * lane_id() + 1u < cnt) {
        a.ent_u[list][i0 + 1] = u1;
        a.ent_pos[list][i0 + 1] = p1;
        a.ent_row[list][i0 + 1] = r1;
    }
    // blocks b with b * kBlk in [p, p + d): b in [ceil(p / kBlk), floor((p + d - 1) / kBlk)]
    uint32_t bl0 = (p0 + kBlk - 1) / kBlk, c0 = 0, bl1 = (p1 + kBlk - 1) / kBlk, c1 = 0;
    if (d0) {
        const uint32_t bh = (p0 + d0 - 1) / kBlk;
        c0 = bh >= bl0 ? bh - bl0 + 1 : 0u;
    }
    if (d1) {
        const uint32_t bh = (p1 + d1 - 1) / kBlk;
        c1 = bh >= bl1 ? bh - bl1 + 1 : 0u;
    }
    const uint32_t bc = c0 + c1;
    const uint32_t binc = warp_incl_scan(bc);
    const uint32_t btot = __shfl_sync(0xffffffffu, binc, 31);
    uint32_t *bf = a.blk_first[list];
    for (uint32_t tb = 0; tb < btot; tb += 32) {
        const uint32_t t = tb + lane_id();
        const int o = owner_of(binc, t);
        const int src = t < btot ? o : 0;
        const uint32_t oinc = __shfl_sync(0xffffffffu, binc, src);
        const uint32_t obc = __shfl_sync(0xffffffffu, bc, src);
        const uint32_t oc0 = __shfl_sync(0xffffffffu, c0, src);
        const uint32_t obl0 = __shfl_sync(0xffffffffu, bl0, src);
        const uint32_t obl1 = __shfl_sync(0xffffffffu, bl1, src);
        if (t < btot) {
            const uint32_t r = t - (oinc - obc);
            const uint32_t ent = E0 + 2u * (uint32_t)src + (r < oc0 ? 0u : 1u);
            const uint32_t b = r < oc0 ? obl0 + r : obl1 + (r - oc0);
            bf[b] = ent;
        }
    }
}

// Moves a warp's staged appends to list `list`.  Warp-collective; st_n warp-uniform.
__device__ __forceinline__ void stage_publish(const LbArgs &a, LbStage &st, uint32_t &st_n, uint32_t list,
                                              unsigned long long *cursor) {
    if (st_n == 0) return;
    __syncwarp();
    const uint32_t i0 = 2u * lane_id(), i1 = i0 + 1u;
    const bool h0 = i0 < st_n, h1 = i1 < st_n;
    publish(a, list, cursor, st_n, h0 ? st.u[i0] : 0, h0 ? st.deg[i0] : 0u, h0 ? st.row[i0] : 0,
            h1 ? st.u[i1] : 0, h1 ? st.deg[i1] : 0u, h1 ? st.row[i1] : 0);
    __syncwarp();
    st_n = 0;
}

// The advances of one slot of the warp: improved[lane] for vertex v.  In list mode
// the first setter of v's bit in B_{k+1} appends v (with its degree and row).
// Warp-collective.
__device__ __forceinline__ void stage_new(const LbArgs &a, bool newly, int32_t v, uint32_t deg, int32_t row,
                                          LbStage &st, uint32_t &st_n, uint32_t list, unsigned long long *cursor) {
    const uint32_t bal = __ballot_sync(0xffffffffu, newly);
    if (!bal) return;
    const uint32_t cnt = __popc(bal);
    if (st_n + cnt > kLbStage) stage_publish(a, st, st_n, list, cursor);
    if (newly) {
        const uint32_t slot = st_n + __popc(bal & lanemask_lt());
        st.u[slot] = v;
        st.deg[slot] = deg;
        st.row[slot] = row;
    }
    __syncwarp();
    st_n += cnt;
}

// One block of kBlk arc positions of list `cur` (entries E, arcs A): relax every
// arc whose source entry is not skipped.  Returns the arcs examined (lane 0).
template <bool UNIT>
__device__ __forceinline__ uint32_t lb_block(const LbArgs &a, uint32_t b, uint32_t E, uint32_t A, uint32_t cur,
                                             uint32_t *bm_next, bool dense_next, LbStage &st, uint32_t &st_n,
                                             unsigned long long *ncursor, uint32_t &adv, uint32_t &items) {
    const uint32_t base = b * kBlk;
    const uint32_t bend = min(base + kBlk, A);
    uint32_t e0 = __ldcg(a.blk_first[cur] + b);
    uint32_t done = base, examined = 0;
    const int32_t *eu = a.ent_u[cur];
    const uint32_t *ep = a.ent_pos[cur];
    const int32_t *er = a.ent_row[cur];
    while (done < bend) {
        // the entries e0 .. e0 + 31 (one per lane) and where the window ends
        const uint32_t ent = e0 + lane_id();
        const bool have = ent < E;
        uint32_t p_l = 0xFFFFFFFFu, du_l = 0;
        int32_t r_l = 0, u_l = 0;
        if (have) {
            p_l = __ldcg(ep + ent);
            r_l = __ldcg(er + ent);
            u_l = __ldcg(eu + ent);
        }
        uint32_t stop = bend, nxt = 0xFFFFFFFFu;
        if (e0 + 32u < E) {
            if (lane_id() == 0) nxt = __ldcg(ep + e0 + 32u);
            nxt = __shfl_sync(0xffffffffu, nxt, 0);
            stop = min(bend, nxt);
        }
        // q_l: where lane l's entry ends (the next entry's start); the owner of
        // position p is the number of lanes with q_l <= p
        uint32_t q_l = __shfl_down_sync(0xffffffffu, p_l, 1);
        if (lane_id() == 31) q_l = nxt;
        bool skip_l = true;
        if (have && p_l < stop) {
            // entries that own no position of [done, stop) need no state
            du_l = __ldcg(a.dist + u_l);
            const uint32_t nb = __ldcg(bm_next + (u_l >> 5));
            skip_l = ((nb >> (u_l & 31)) & 1u) != 0;
        }
        // the first owner may start before `done` (it is e0 or the window's first entry)
        items += (have && !skip_l && p_l >= done && p_l < stop) ? 1u : 0u;
        int32_t v[kLbU];
        uint32_t cand[kLbU];
        bool ok[kLbU];
#pragma unroll
        for (int j = 0; j < kLbU; j++) {
            const uint32_t p = done + 32u * j + lane_id();
            const int src = owner_of(q_l, p);
            const uint32_t po = __shfl_sync(0xffffffffu, p_l, src);
            const int32_t ro = __shfl_sync(0xffffffffu, r_l, src);
            const uint32_t dq = __shfl_sync(0xffffffffu, du_l, src);
            const bool sk = __shfl_sync(0xffffffffu, skip_l, src);
            ok[j] = p < stop && !sk;
            v[j] = 0;
            uint32_t w = 0;
            if (ok[j]) {
                const uint32_t e = (uint32_t)ro + (p - po);
                v[j] = __ldcs(a.idx + e);
                w = UNIT ? 1u : __ldcs(a.w + e);
            }
            cand[j] = dq + w;
            if (ok[j] && (cand[j] < dq || cand[j] == kInf)) {
                set_status(a.h, LLP_ERR_OVERFLOW);
                ok[j] = false;
            }
        }
        uint32_t dv[kLbU];
#pragma unroll
        for (int j = 0; j < kLbU; j++) dv[j] = ok[j] ? __ldcg(a.dist + v[j]) : 0u;
        bool imp[kLbU];
        bool any = false;
#pragma unroll
        for (int j = 0; j < kLbU; j++) {
            examined += ok[j] ? 1u : 0u;
            imp[j] = ok[j] && cand[j] < dv[j];
            if (imp[j]) red_min_u32(a.dist + v[j], cand[j]);
            adv += imp[j] ? 1u : 0u;
            any |= imp[j];
        }
        if (__any_sync(0xffffffffu, any)) {
            if (dense_next) {
#pragma unroll
                for (int j = 0; j < kLbU; j++)
                    if (imp[j]) red_or_u32(bm_next + (v[j] >> 5), 1u << (v[j] & 31));
            } else {
                uint32_t old[kLbU];
                int32_t o0[kLbU], o1[kLbU];
#pragma unroll
                for (int j = 0; j < kLbU; j++) {
                    old[j] = 0;
                    o0[j] = 0;
                    o1[j] = 0;
                    if (imp[j]) {
                        old[j] = atomicOr(bm_next + (v[j] >> 5), 1u << (v[j] & 31));
                        o0[j] = __ldg(a.off + v[j]);
                        o1[j] = __ldg(a.off + v[j] + 1);
                    }
                }
#pragma unroll
                for (int j = 0; j < kLbU; j++) {
                    const bool nw = imp[j] && ((old[j] >> (v[j] & 31)) & 1u) == 0 && o1[j] > o0[j];
                    stage_new(a, nw, v[j], (uint32_t)(o1[j] - o0[j]), o0[j], st, st_n, cur ^ 1u, ncursor);
                }
            }
        }
        const uint32_t nd = min(done + kBlk, stop);
        if (nd >= stop && stop < bend) e0 += 32u;
        done = nd;
    }
    return warp_sum(examined);
}

// Turns the bitmap B (bit v set: v was advanced) into the entry list `list`,
// vertices without out-arcs left out, and clears B.  CTA b takes a contiguous
// range of bitmap words, each of its warps a contiguous sub-range; a first pass
// counts entries and arcs, one atomic add per CTA reserves them, a second pass
// writes them.  Every thread of the CTA calls it.
__device__ void lb_compact(const LbArgs &a, uint32_t *B, uint32_t list, unsigned long long *cursor,
                           unsigned long long *s_wtot, unsigned long long *s_base) {
    const int wid = threadIdx.x >> 5;
    const int64_t nw = a.nwords;
    const int64_t c0 = nw * blockIdx.x / gridDim.x, c1 = nw * (blockIdx.x + 1) / gridDim.x;
    const int64_t w0 = c0 + (c1 - c0) * wid / kLbWarps, w1 = c0 + (c1 - c0) * (wid + 1) / kLbWarps;
    // pass 1: count
    uint32_t cnt = 0, arcs = 0;
    for (int64_t wb = w0; wb < w1; wb += kCompactWords) {
        uint32_t d[kCompactWords];
#pragma unroll
        for (int j = 0; j < kCompactWords; j++) {
            d[j] = 0;
            const int64_t wi = wb + j;
            if (wi < w1) {
                const uint32_t word = __ldcg(B + wi);
                const int64_t v = wi * 32 + lane_id();
                if ((word >> lane_id()) & 1u) d[j] = (uint32_t)(__ldg(a.off + v + 1) - __ldg(a.off + v));
            }
        }
#pragma unroll
        for (int j = 0; j < kCompactWords; j++) {
            cnt += d[j] ? 1u : 0u;
            arcs += d[j];
        }
    }
    cnt = warp_sum(cnt);
    arcs = warp_sum(arcs);
    if (lane_id() == 0) s_wtot[wid] = ((unsigned long long)cnt << 32) | arcs;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tot = 0;
        for (int i = 0; i < kLbWarps; i++) {
            const unsigned long long x = s_wtot[i];
            s_wtot[i] = tot;
            tot += x;
        }
        *s_base = tot ? atomicAdd(cursor, tot) : 0ull;
    }
    __syncthreads();
    const unsigned long long wb0 = *s_base + s_wtot[wid];
    uint32_t E = (uint32_t)(wb0 >> 32), P = (uint32_t)wb0;
    // pass 2: write entries in word order, lanes in vertex order; clear the words
    uint32_t *bf = a.blk_first[list];
    for (int64_t wb = w0; wb < w1; wb += kCompactWords) {
        uint32_t d[kCompactWords];
        int32_t r[kCompactWords];
#pragma unroll
        for (int j = 0; j < kCompactWords; j++) {
            d[j] = 0;
            r[j] = 0;
            const int64_t wi = wb + j;
            if (wi < w1) {
                const uint32_t word = __ldcg(B + wi);
                const int64_t v = wi * 32 + lane_id();
                if ((word >> lane_id()) & 1u) {
                    r[j] = __ldg(a.off + v);
                    d[j] = (uint32_t)(__ldg(a.off + v + 1) - r[j]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kCompactWords; j++) {
            const int64_t wi = wb + j;
            const bool has = d[j] > 0;
            const uint32_t bal = __ballot_sync(0xffffffffu, has);
            const uint32_t incl = warp_incl_scan(d[j]);
            const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
            const uint32_t p = P + incl - d[j];
            if (has) {
                const uint32_t i = E + __popc(bal & lanemask_lt());
                a.ent_u[list][i] = (int32_t)(wi * 32 + lane_id());
                a.ent_pos[list][i] = p;
                a.ent_row[list][i] = r[j];
                // blocks whose first arc position lies in [p, p + d)
                const uint32_t bl = (p + kBlk - 1) / kBlk, bh = (p + d[j] - 1) / kBlk;
                for (uint32_t b = bl; b <= bh && bh >= bl; b++) bf[b] = i;
            }
            E += __popc(bal);
            P += tot;
            if (lane_id() == 0 && wi < w1) B[wi] = 0u;
        }
    }
}

template <bool UNIT>
__global__ void __launch_bounds__(kLbThreads, 2) lb_sweep_kernel(LbArgs a) {
    __shared__ LbStage s_stage[kLbWarps];
    __shared__ uint32_t s_work[2];
    __shared__ unsigned long long s_edges;
    __shared__ unsigned long long s_wtot[kLbWarps];
    __shared__ unsigned long long s_base;
    WsHeader *h = a.h;
    const long long t0 = globaltimer_ns();
    const long long deadline = t0 + a.deadline_ns;
    uint32_t phase = 0;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
    const int wid = threadIdx.x >> 5;
    LbStage &st = s_stage[wid];
    uint32_t st_n = 0;
    unsigned long long *cur3 = h->lb_cursor;
    if (threadIdx.x == 0) {
        s_work[0] = 0;
        s_work[1] = 0;
        s_edges = 0;
    }

    // ---- init_global_state (paper Sec. 3.3): d = infinity except the source
    // (a warm start keeps the caller's dist[]); both bitmaps cleared
    for (int64_t v = gtid; v < a.n; v += gthreads)
        if (!a.warm || v == a.source) a.dist[v] = (v == a.source) ? 0u : kInf;
    for (int64_t wi = gtid; wi < a.nwords; wi += gthreads) {
        a.bm[0][wi] = 0u;
        a.bm[1][wi] = 0u;
    }
    if (gtid == 0) {
        h->t_start = t0;
        h->mode_used = a.mode;
        h->delta_used = kInf;
        h->block_cfg_used = 4;
    }
    bool alive = grid_barrier(h, phase, deadline);

    // ---- initial_states_to_process: list 1 = the source (cold) or the seeds (warm)
    if (alive) {
        if (!a.warm) {
            const int32_t s0 = __ldg(a.off + a.source), s1 = __ldg(a.off + a.source + 1);
            const uint32_t deg = (uint32_t)(s1 - s0);
            if (deg > 0) {
                if (gtid == 0) {
                    a.ent_u[1][0] = a.source;
                    a.ent_pos[1][0] = 0;
                    a.ent_row[1][0] = s0;
                    cur3[1] = (1ull << 32) | deg;
                }
                for (int64_t b = gtid; b < (int64_t)((deg + kBlk - 1) / kBlk); b += gthreads) a.blk_first[1][b] = 0u;
            }
        } else {
            const int64_t gw = gtid >> 5, nwp = gthreads >> 5;
            for (int64_t base = gw * 32; base < a.n_seeds; base += nwp * 32) {
                const int64_t i = base + lane_id();
                int32_t u = i < a.n_seeds ? a.seeds[i] : -1;
                if (i < a.n_seeds && (uint32_t)u >= (uint32_t)a.n) {
                    set_status(h, LLP_ERR_INVALID_ARG);
                    u = -1;
                }
                bool nw = false;
                int32_t r0 = 0;
                uint32_t deg = 0;
                if (u >= 0) {
                    r0 = __ldg(a.off + u);
                    deg = (uint32_t)(__ldg(a.off + u + 1) - r0);
                    if (deg > 0 && __ldcg(a.dist + u) != kInf) {
                        const uint32_t bit = 1u << (u & 31);
                        nw = (atomicOr(a.bm[1] + (u >> 5), bit) & bit) == 0;
                    }
                }
                stage_new(a, nw, u, deg, r0, st, st_n, 1u, &cur3[1]);
            }
            stage_publish(a, st, st_n, 1u, &cur3[1]);
        }
    }
    if (alive) alive = grid_barrier(h, phase, deadline);

    uint32_t k = 1, dense_sweeps = 0;
    uint32_t adv = 0, items = 0;
    bool prev_dense = false;
    while (alive) {
        const unsigned long long cv = *(volatile unsigned long long *)&cur3[k % 3];
        const uint32_t E = (uint32_t)(cv >> 32), A = (uint32_t)cv;
        if (gtid == 0) {
            cur3[(k + 2) % 3] = 0ull;  // list k - 1's cursor: read by nobody in sweep k
            if (k - 1 < kSweepLogCap)
                sweep_log(h)[k - 1] = SweepRec{(uint32_t)(globaltimer_ns() - t0), E, A, (prev_dense ? 1u : 0u)};
            const unsigned long long pe = *(volatile unsigned long long *)&h->sweep_edges[(k - 1) & 1];
            h->sweep_edges[(k - 1) & 1] = 0;
            if (k >= 2 && k - 2 < kSweepLogCap) {
                const unsigned long long q = min(pe >> 10, 0x3FFFFFFFull);
                sweep_log(h)[k - 2].flags |= (uint32_t)(q << 2);
            }
        }
        if (A == 0) break;
        dense_sweeps += prev_dense ? 1u : 0u;
        const bool dense_next =
            a.mode == LLP_MODE_DENSE || (a.mode == LLP_MODE_AUTO && (unsigned long long)A > a.dense_arcs);
        const uint32_t cur = k & 1u;
        uint32_t *bm_next = a.bm[cur ^ 1u];
        if (!prev_dense) {
            // B_k deduplicated list k's appends; nobody reads it in this sweep
            uint32_t *bc = a.bm[cur];
            for (int64_t wi = gtid; wi < a.nwords; wi += gthreads) bc[wi] = 0u;
        }
        if (threadIdx.x == 0) s_work[(k + 1) & 1] = 0;  // used after the next grid barrier
        const uint32_t nblk = (A + kBlk - 1) / kBlk;
        uint32_t examined = 0;
        for (;;) {
            uint32_t j = 0;
            if (lane_id() == 0) j = atomicAdd(&s_work[k & 1], 1u);
            j = __shfl_sync(0xffffffffu, j, 0);
            const uint64_t b = (uint64_t)blockIdx.x + (uint64_t)j * gridDim.x;
            if (b >= nblk) break;
            examined += lb_block<UNIT>(a, (uint32_t)b, E, A, cur, bm_next, dense_next, st, st_n,
                                       &cur3[(k + 1) % 3], adv, items);
        }
        stage_publish(a, st, st_n, cur ^ 1u, &cur3[(k + 1) % 3]);
        if (lane_id() == 0 && examined) atomicAdd(&s_edges, (unsigned long long)examined);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (s_edges) {
                atomicAdd(&h->sweep_edges[k & 1], s_edges);
                atomicAdd(&h->edges, s_edges);
            }
            s_edges = 0;
        }
        alive = grid_barrier(h, phase, deadline);
        if (alive && dense_next) {
            lb_compact(a, bm_next, cur ^ 1u, &cur3[(k + 1) % 3], s_wtot, &s_base);
            alive = grid_barrier(h, phase, deadline);
        }
        prev_dense = dense_next;
        k += 1;
    }

    // ---- final_solution: dist[] already holds G; statistics (one atomic per warp)
    const unsigned long long it_s = warp_sum((unsigned long long)items), ad_s = warp_sum((unsigned long long)adv);
    if (lane_id() == 0) {
        atomicAdd(&h->items, it_s);
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

}  // namespace

size_t lb_workspace_bytes(int32_t n, int64_t m) {
    const size_t nblk = (size_t)(m / kBlk) + 2;
    return 2 * (3 * align_up((size_t)n * 4, 256) + align_up(nblk * 4, 256));
}

// Carves the load-balanced engine's lists from `base` (256-byte aligned).
static void lb_carve(char *base, int32_t n, int64_t m, LbArgs &a) {
    const size_t nblk = (size_t)(m / kBlk) + 2;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base + off;
        off += align_up(bytes, 256);
        return p;
    };
    for (int l = 0; l < 2; l++) {
        a.ent_u[l] = (int32_t *)take((size_t)n * 4);
        a.ent_pos[l] = (uint32_t *)take((size_t)n * 4);
        a.ent_row[l] = (int32_t *)take((size_t)n * 4);
        a.blk_first[l] = (uint32_t *)take(nblk * 4);
    }
}

llp_status_t lb_launch(bool unit, const llp_csr_t *g, int32_t source, uint32_t *dist, uint32_t *bm0, uint32_t *bm1,
                       void *lists, WsHeader *h, long long deadline_ns, int32_t mode, unsigned long long dense_arcs,
                       const int32_t *seeds, int32_t n_seeds, cudaStream_t stream) {
    LbArgs a{};
    a.n = g->n;
    a.source = source;
    a.nwords = (int32_t)(((int64_t)g->n + 31) / 32);
    a.off = (const int32_t *)g->offsets;
    a.idx = g->indices;
    a.w = unit ? nullptr : g->weights;
    a.dist = dist;
    a.bm[0] = bm0;
    a.bm[1] = bm1;
    lb_carve((char *)lists, g->n, g->m, a);
    a.h = h;
    a.deadline_ns = deadline_ns;
    a.dense_arcs = dense_arcs;
    a.mode = mode;
    a.warm = n_seeds >= 0 ? 1 : 0;
    a.n_seeds = n_seeds > 0 ? n_seeds : 0;
    a.seeds = seeds;
    void *kargs[] = {&a};
    const int max_blocks = (int)std::max<int64_t>(32, ((int64_t)g->n + 1023) / 1024);
    const void *fn = unit ? (const void *)lb_sweep_kernel<true> : (const void *)lb_sweep_kernel<false>;
    return launch_cooperative(fn, kLbThreads, 0, max_blocks, kargs, stream);
}

}  // namespace llp

// Persistent forbidden/advance sweep engine for the graph problems:
// SSSP (paper Sec. 4.1) and BFS (paper Sec. 4.2).
//
// State G[v] = d(v) (uint32, 0xFFFFFFFF = "infinity"), kept during the run in
// the caller's dist[] itself (no copy at the end).  A vertex v is forbidden
// when some arc (u, v) offers d(u) + w(u, v) < d(v); the advance lowers d(v)
// with an atomic min, the lock-free monotone update whose requirements the
// paper lists in Sec. 3.2 (atomic, monotone, progress detection).  The
// predicate is evaluated push-style: when u is taken from the worklist each
// out-arc is checked, and every advance makes v a candidate of the next sweep
// (the paper's problem-specific state selection, Sec. 3.2).
//
// One cooperative launch runs all sweeps, separated by a bounded grid barrier.
//   - the worklist of sweep k is a bitmap B_k (one bit per vertex, three
//     buffers used in turn, B_k = bm[k mod 3]); atomicOr on B_{k+1}
//     deduplicates advances, and a push sweep k clears B_k as it reads it, so
//     B_k is clean when it becomes B_{k+3};
//   - a per-vertex class (1: small, out-degree <= small_max; 2: large; 0: no
//     out-arcs), computed once per call into a per-32-vertex table, routes
//     advanced vertices: large ones go to a chunk list (chunks of chunk_edges
//     arcs, one per warp, so hubs spread over the grid), small ones either to a
//     list (sparse sweep, warp-aggregated appends) or only to the bitmap (dense
//     sweep: fire-and-forget atomicOr, the next sweep scans the bitmap like the
//     paper's all-indices solver, without any shared counter in the hot loop);
//   - small vertices are expanded 32 per warp, arcs balanced across the lanes,
//     kUnroll arcs per lane in flight (the random reads of d(v) are the
//     bottleneck; they need many independent loads per lane to reach the
//     device's random-access rate);
//   - the advance itself is a fire-and-forget atomic min on dist[v] issued
//     when the candidate beats the value just read (a stale read only costs a
//     redundant visit: distances only decrease); the advanced targets wait in
//     a per-warp buffer and enter the next worklist in bulk (class lookup,
//     bitmap dedup, appends), so a batch of arcs ends at the read of d(v);
//   - the per-CTA state of the run (schedule, bucket bounds, bitmap pointers,
//     sweep flags) lives in shared memory, written by one thread per sweep,
//     and one thread per CTA reads the sweep's worklist sizes: registers stay
//     free for the arcs in flight;
//   - with a finite bucket width delta (the paper's bucket worklist, Sec. 3.3)
//     only advances with d below the current bucket bound enter the next
//     worklist; the others wait in a far list filtered when the near worklist
//     empties.
// The run stops when no index is forbidden: every worklist is empty.
//
// BFS with the transpose (llp_bfs_pull) may evaluate a wide sweep pull-style:
// every vertex not reached yet scans its in-arcs and stops at the first source
// in the frontier bitmap.  Such a sweep reads the frontier at random, so it
// cannot clear it as it goes; three bitmaps rotate by sweep (k mod 3) and the
// one a pull sweep left behind is cleared during the following sweep, which
// neither reads nor writes it.
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "llp_common.cuh"
#include "sweep_init.cuh"

namespace llp {

template <typename OffT>
llp_status_t enqueue_learned_prologue(const llp_csr_t *g, int32_t source, bool unit, const float *params, WsHeader *h,
                                      const SweepInit<OffT> &init, cudaStream_t st);
size_t lb_workspace_bytes(int32_t n, int64_t m);
llp_status_t lb_launch(bool unit, const llp_csr_t *g, int32_t source, uint32_t *dist, uint32_t *bm0, uint32_t *bm1,
                       void *lists, WsHeader *h, long long deadline_ns, int32_t mode, unsigned long long dense_arcs,
                       const int32_t *seeds, int32_t n_seeds, cudaStream_t stream);

namespace {

struct BlockCfg {
    int small_max;
    int chunk;
};
// (small-vertex out-degree limit, arcs per chunk of a large vertex); vertices
// just above the limit cost a whole warp each, so the default keeps degrees up
// to 64 in the lane-balanced 32-vertex groups.
__host__ __device__ inline BlockCfg block_cfg_of(int c) {
    return c == 1 ? BlockCfg{32, 256} : (c == 3 ? BlockCfg{128, 512} : BlockCfg{64, 256});
}

#ifndef LLP_SWEEP_UNROLL
#define LLP_SWEEP_UNROLL 4
#endif
#ifndef LLP_SWEEP_MIN_BLOCKS
#define LLP_SWEEP_MIN_BLOCKS 2
#endif
constexpr int kUnroll = LLP_SWEEP_UNROLL;  // arcs per lane in flight (push sweeps)
constexpr int kPullUnroll = 4;  // in-arcs per lane and round (pull sweeps)
#ifndef LLP_DENSE_GROUP_WORDS
#define LLP_DENSE_GROUP_WORDS 8
#endif
constexpr int kGroupWords = LLP_DENSE_GROUP_WORDS;  // bitmap words per dense-sweep item
// A hub source whose 256-arc chunks would not give every warp one is seeded as
// chunks of kFineChunk arcs (chunk index | kFineFlag in the list entry).
constexpr int32_t kFineChunk = 64;
constexpr int32_t kFineFlag = 1 << 30;
#ifndef LLP_ONE_BUCKET_FAST
#define LLP_ONE_BUCKET_FAST 1
#endif
#ifndef LLP_MIN_GROUP
#define LLP_MIN_GROUP 4
#endif
// A sparse sweep whose worklist would not give every warp a group of 32 vertices
// takes groups of 16, 8, ... down to kMinGroup vertices (their arcs still spread
// over the 32 lanes), so the few busy warps run shorter chains.
constexpr uint32_t kMinGroup = LLP_MIN_GROUP;
#ifndef LLP_CTAKE
#define LLP_CTAKE 4
#endif
#ifndef LLP_CTAKE_MIN
#define LLP_CTAKE_MIN 24
#endif
constexpr uint32_t kTake = LLP_CTAKE;        // chunk items per claim in wide chunk sweeps
constexpr uint32_t kTakeMin = LLP_CTAKE_MIN;  // ... with at least this many per warp

template <typename OffT>
struct GraphArgs {
    int32_t n;
    int32_t source;
    int32_t nwords;  // ceil(n / 32)
    const OffT *off;
    const int32_t *idx;
    const uint32_t *w;
    uint32_t *dist;                 // state during the run, and the output
    uint2 *cls;      // per 32 vertices: x = has out-arcs, y = large
    uint32_t *bm[3]; // frontier bitmaps, B_k = bm[k % 3]
    // pull sweeps (BFS only): in-arcs, visited bitmap, frontier size that selects them
    const OffT *in_off;              // NULL: push only
    const int32_t *in_idx;
    uint32_t *vis;                   // valid after a pull sweep: bit set = level known
    unsigned long long pull_arcs;
    int32_t *small[2];
    int2 *chunk[2];
    int2 *far[2];
    uint32_t far_cap;
    uint32_t *trace;  // LLP_SWEEP_TRACE builds only: per sweep and CTA, first-warp and CTA finish times
    uint32_t *fixed;  // fixed-state memoization (NULL: off): bit v set = d(v) is final
    WsHeader *h;
    uint32_t delta;  // kInf: no buckets
    int32_t mode;
    unsigned long long dense_arcs;  // AUTO: dense next sweep when this sweep's arcs exceed it
    int32_t small_max;
    int32_t chunk_edges;
    int32_t cfg;
    int32_t use_dev_sched;  // 1: take mode/delta/cfg from the header (learned scheduler)
    int32_t pre_init;       // 1: the state was initialised by the learned scheduler's prologue
    int32_t local_chain;    // batches per worklist item of the local chain, 0 = off
    int32_t group_words;    // dense sweeps: bitmap words per item (1, 2, 4, 8), 0 = from the grid size
    long long deadline_ns;
    // warm start: G starts from dist[] (upper bounds of the distances) and the first
    // worklist is seeds[0..n_seeds) instead of the source alone
    int32_t warm;
    int32_t n_seeds;
    const int32_t *seeds;
};

// Buffer selection by sweep parity / rotation without indexing the parameter
// arrays with a run-time value (which would copy the arguments to the stack).
template <typename T>
__device__ __forceinline__ T *pick2(T *const (&arr)[2], uint32_t i) { return (i & 1u) ? arr[1] : arr[0]; }
template <typename T>
__device__ __forceinline__ T *pick3(T *const (&arr)[3], uint32_t i) {
    const uint32_t r = i % 3u;
    return r == 0 ? arr[0] : (r == 1 ? arr[1] : arr[2]);
}

// Per-thread (mostly warp-uniform) state of a run.
struct SweepCtx {
    uint32_t k;                    // current sweep
    uint32_t lq_n = 0;             // entries on the warp's local-chain stack
    bool chain_on = false;         // the local chain is active in this warp
    uint32_t items = 0, adv = 0;   // statistics of the run
    uint32_t edges = 0;            // arcs examined in this sweep (lane 0 mostly)
    uint32_t marked = 0;           // dense_next marks (an upper bound of the next frontier)
    uint32_t st_ns = 0, st_nc = 0; // staged worklist appends of the warp (warp-uniform)
    uint32_t pend_n = 0;           // deferred advances in g_pend (warp-uniform)
};

// Per-CTA state of a run that every thread reads: written by thread 0 at the
// start of the run and of each sweep, read after a CTA barrier.  Keeping it in
// shared memory keeps the sweep's registers for the arcs in flight.
struct SweepShared {
    unsigned long long bucket_hi;  // exclusive bound of the current bucket
    unsigned long long fixed_lo;   // every d below it is final (the previous bucket's bound)
    unsigned long long next_hi;    // bound of the next bucket (taken at the start of the next sweep)
    uint32_t *bm_cur, *bm_next;    // B_k and B_{k+1}
    int32_t mode, cfg, small_max, chunk_edges;
    int32_t gw;                    // dense sweeps: bitmap words per item
    int32_t chain;                 // batches of 32 a warp may take from its stack per worklist item
    uint32_t delta;
    uint32_t fa;                   // far-list generation
    uint32_t ns, nc, nf, fmin;     // sizes of the sweep's worklists, far list and its least candidate
    bool dense;                    // this sweep scans B_k
    bool dense_next;               // small advances only set their bitmap bit
    bool pull;                     // this sweep runs over the in-arcs
    bool prev_pull;                // the previous sweep ran over the in-arcs
    bool vis_valid;                // a.vis holds every vertex reached so far
    bool advance_bucket;           // the next sweep starts the bucket next_hi
    bool fine_src;                 // the source is seeded as chunks of kFineChunk arcs
    uint32_t gsz;                  // sparse sweep: list entries per vertex group (kMinGroup..32)
};


constexpr uint32_t kStageSmall = 128;  // entries per warp
constexpr uint32_t kStageChunk = 128;
constexpr uint32_t kDirectChunks = 4;  // a lane with more chunk entries reserves them directly
constexpr uint32_t kLocalQ = 128;      // per-warp stack of the local chain
// after a flush a warp stages at most 32 lanes x kUnroll small vertices, or 32 lanes x
// kDirectChunks chunk entries, at once
static_assert(kStageSmall >= 32 * kUnroll && kStageChunk >= 32 * kDirectChunks, "staging buffers too small");

__shared__ SweepShared g_sh;
__shared__ int32_t g_stage_small[16][kStageSmall];  // per warp
__shared__ int2 g_stage_chunk[16][kStageChunk];
__shared__ int32_t g_lq[16][kLocalQ];
// Deferred worklist insertion: a relaxation that advances v only issues the atomic
// min and records v in its warp's buffer; the class lookup and the bitmap/list
// insertion of the buffered targets run in bulk once kPendT of them are pending
// (and at the end of the sweep), so a batch's chain of dependent loads ends at
// the read of d(v).  The "advanced again" bits of the next frontier are set later
// than the advance itself, which lets a few more stale vertices be expanded.
#ifndef LLP_DEFER
#define LLP_DEFER 64
#endif
constexpr uint32_t kPendT = LLP_DEFER;
constexpr uint32_t kPendCap = kPendT + 32 * kUnroll;  // at most kPendT - 1 + one batch
__shared__ int32_t g_pend[16][kPendCap];
__device__ __forceinline__ int warp_in_cta() { return threadIdx.x >> 5; }

// Moves a warp's staged entries to the global list (one reservation).
template <typename T>
__device__ __forceinline__ void stage_flush(T *stage, uint32_t &cnt, T *list, uint32_t *counter) {
    if (cnt == 0) return;
    __syncwarp();
    uint32_t base = 0;
    if (lane_id() == 0) base = atomicAdd(counter, cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (uint32_t i = lane_id(); i < cnt; i += 32) list[base + i] = stage[i];
    __syncwarp();
    cnt = 0;
}

__device__ __forceinline__ void red_or(uint32_t *p, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.or.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_and(uint32_t *p, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.and.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_min32(uint32_t *p, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.min.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Class of v (0: no out-arcs, 1: small, 2: large) from the per-32-vertex table.
template <typename OffT>
__device__ __forceinline__ uint32_t class_of(const GraphArgs<OffT> &a, int32_t v) {
    const uint2 cw = __ldg(&a.cls[(uint32_t)v >> 5]);
    const uint32_t bit = 1u << (v & 31);
    return (cw.x & bit) ? ((cw.y & bit) ? 2u : 1u) : 0u;
}

// Append the vertices v[j] that entered the frontier bitmap of sweep k+1 for
// the first time (newly[j]) to the small-vertex list or, as chunks, to the
// chunk list of sweep k+1, through the warp's staging buffers.  Warp-collective.
template <typename OffT, int U>
__device__ __forceinline__ void append_new(const GraphArgs<OffT> &a, const bool (&newly)[U], const int32_t (&v)[U],
                                           const uint32_t (&cls)[U], SweepCtx &c) {
    uint32_t n_small = 0, n_large = 0;
    uint32_t nch[U];
#pragma unroll
    for (int j = 0; j < U; j++) {
        nch[j] = 0;
        n_small += (newly[j] && cls[j] == 1);
        if (newly[j] && cls[j] == 2) {
            const uint32_t deg = (uint32_t)(__ldg(a.off + v[j] + 1) - __ldg(a.off + v[j]));
            nch[j] = (deg + g_sh.chunk_edges - 1) / g_sh.chunk_edges;
            n_large += nch[j];
        }
    }
    const uint32_t nk = c.k + 1;
    const uint32_t nx = nk % 3;
    if (__any_sync(0xffffffffu, n_small > 0)) {
        uint32_t incl = n_small;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane_id() >= o) incl += t;
        }
        const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
        if (c.st_ns + tot > kStageSmall) stage_flush(g_stage_small[warp_in_cta()], c.st_ns, pick2(a.small, nk), &a.h->n_small[nx]);
        uint32_t slot = c.st_ns + incl - n_small;
#pragma unroll
        for (int j = 0; j < U; j++)
            if (newly[j] && cls[j] == 1) g_stage_small[warp_in_cta()][slot++] = v[j];
        c.st_ns += tot;
    }
    if (__any_sync(0xffffffffu, n_large > 0)) {
        // lanes with many chunks (vertices of degree > kDirectChunks*chunk) reserve directly
        const bool direct = n_large > kDirectChunks;
        if (__any_sync(0xffffffffu, direct)) {
            uint32_t slot = warp_reserve(direct ? n_large : 0u, &a.h->n_chunk[nx]);
            int2 *dst = pick2(a.chunk, nk);
            if (direct) {
#pragma unroll
                for (int j = 0; j < U; j++)
                    for (uint32_t q = 0; q < nch[j]; q++) dst[slot++] = make_int2(v[j], (int)q);
            }
        }
        const uint32_t mine = direct ? 0u : n_large;
        uint32_t incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane_id() >= o) incl += t;
        }
        const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
        if (tot) {
            if (c.st_nc + tot > kStageChunk) stage_flush(g_stage_chunk[warp_in_cta()], c.st_nc, pick2(a.chunk, nk), &a.h->n_chunk[nx]);
            uint32_t slot = c.st_nc + incl - mine;
            if (!direct) {
#pragma unroll
                for (int j = 0; j < U; j++)
                    for (uint32_t q = 0; q < nch[j]; q++) g_stage_chunk[warp_in_cta()][slot++] = make_int2(v[j], (int)q);
            }
            c.st_nc += tot;
        }
    }
}

// Put the advanced vertices v[j] (want[j], class cls[j]) into the worklist of
// sweep k+1, all kUnroll of them at once.  Warp-collective.
template <typename OffT, int U>
__device__ __forceinline__ void push_near(const GraphArgs<OffT> &a, const bool (&want_in)[U], const int32_t (&v)[U],
                                          const uint32_t (&cls)[U], SweepCtx &c) {
    bool want[U];
#pragma unroll
    for (int j = 0; j < U; j++) want[j] = want_in[j];
    if (c.chain_on) {
        // small advances stay with this warp when its stack has room for all of them
        uint32_t nl = 0;
#pragma unroll
        for (int j = 0; j < U; j++) nl += (want[j] && cls[j] == 1);
        uint32_t incl = nl;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane_id() >= o) incl += t;
        }
        const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
        if (tot > 0 && c.lq_n + tot <= kLocalQ) {
            uint32_t slot = c.lq_n + incl - nl;
#pragma unroll
            for (int j = 0; j < U; j++)
                if (want[j] && cls[j] == 1) {
                    g_lq[warp_in_cta()][slot++] = v[j];
                    want[j] = false;
                }
            c.lq_n += tot;
        }
    }
    bool newly[U];
#pragma unroll
    for (int j = 0; j < U; j++) {
        newly[j] = false;
        if (want[j] && cls[j] != 0) {
            const uint32_t bit = 1u << (v[j] & 31);
            uint32_t *word = g_sh.bm_next + (v[j] >> 5);
            if (g_sh.dense_next && cls[j] == 1) {
                red_or(word, bit);
                c.marked++;
            } else {
                newly[j] = (atomicOr(word, bit) & bit) == 0;
            }
        }
    }
    append_new(a, newly, v, cls, c);
}

// Drains the deferred advances of the warp: the targets collected in g_pend get
// their class and enter the next worklist, kUnroll per lane at a time.
// Warp-collective.
template <typename OffT>
__device__ __forceinline__ void drain_pending(const GraphArgs<OffT> &a, SweepCtx &c) {
    __syncwarp();
    for (uint32_t base = 0; base < c.pend_n; base += 32 * kUnroll) {
        bool want[kUnroll];
        int32_t v[kUnroll];
        uint32_t cls[kUnroll];
#pragma unroll
        for (int j = 0; j < kUnroll; j++) {
            const uint32_t i = base + 32 * j + lane_id();
            want[j] = i < c.pend_n;
            v[j] = want[j] ? g_pend[warp_in_cta()][i] : 0;
        }
#pragma unroll
        for (int j = 0; j < kUnroll; j++) cls[j] = want[j] ? class_of(a, v[j]) : 0u;
        push_near(a, want, v, cls, c);
    }
    __syncwarp();
    c.pend_n = 0;
}

// Evaluate forbidden(v) against candidate distances and advance, for up to
// kUnroll arcs per lane.  cand = d(u) + w(u, v) in 32 bits; ovf marks a sum that
// does not fit (a finite length >= 0xFFFFFFFF).  Warp-collective.
template <typename OffT>
__device__ __forceinline__ void relax_multi(const GraphArgs<OffT> &a, const bool (&ok)[kUnroll],
                                            const int32_t (&v)[kUnroll], const uint32_t (&cand)[kUnroll],
                                            const bool (&ovf)[kUnroll], SweepCtx &c) {
    uint32_t dv[kUnroll];
    bool live[kUnroll];
#pragma unroll
    for (int j = 0; j < kUnroll; j++) live[j] = ok[j];
    if (a.fixed) {
        // fixed-state memoization: a target known to be final is not read
        uint32_t fw[kUnroll];
#pragma unroll
        for (int j = 0; j < kUnroll; j++) fw[j] = ok[j] ? __ldcg(a.fixed + (v[j] >> 5)) : 0u;
#pragma unroll
        for (int j = 0; j < kUnroll; j++) live[j] = ok[j] && ((fw[j] >> (v[j] & 31)) & 1u) == 0;
    }
#pragma unroll
    for (int j = 0; j < kUnroll; j++) dv[j] = live[j] ? __ldcg(a.dist + v[j]) : 0u;
    bool near[kUnroll], far[kUnroll];
    bool any_far = false, any_near = false;
#pragma unroll
    for (int j = 0; j < kUnroll; j++) {
        bool improved = false;
        if (live[j]) {
            if (ovf[j]) {
                set_status(a.h, LLP_ERR_OVERFLOW);
            } else if (cand[j] < dv[j]) {
                red_min32(a.dist + v[j], cand[j]);
                improved = true;
            } else if (a.fixed && (unsigned long long)dv[j] < g_sh.fixed_lo) {
                red_or(a.fixed + (v[j] >> 5), 1u << (v[j] & 31));  // below every pending bucket: final
            }
        }
        c.adv += improved;
        near[j] = improved;
    }
#if LLP_ONE_BUCKET_FAST
    const bool buckets = g_sh.delta != kInf;  // one bucket: every advance is near
#else
    const bool buckets = true;
#endif
    if (buckets) {
#pragma unroll
        for (int j = 0; j < kUnroll; j++) {
            far[j] = near[j] && (unsigned long long)cand[j] >= g_sh.bucket_hi;
            near[j] = near[j] && !far[j];
            any_far |= far[j];
        }
    }
    if (buckets && __any_sync(0xffffffffu, any_far)) {
        uint32_t cnt = 0, fmin = kInf;
#pragma unroll
        for (int j = 0; j < kUnroll; j++) {
            cnt += far[j];
            if (far[j]) fmin = min(fmin, cand[j]);
        }
        uint32_t slot = warp_reserve(cnt, &a.h->n_far[g_sh.fa % 3]);
#pragma unroll
        for (int j = 0; j < kUnroll; j++) {
            if (!far[j]) continue;
            if (slot < a.far_cap) {
                pick2(a.far, g_sh.fa)[slot] = make_int2(v[j], (int)cand[j]);
            } else {
                near[j] = true;  // far list full: keep it in the near worklist (still correct)
            }
            slot++;
        }
        if (cnt) atomicMin(&a.h->far_min[g_sh.fa % 3], fmin);
    }
#if LLP_DEFER
    if (!c.chain_on) {  // with the local chain the advances go to its stack at once
        const uint32_t lt = lanemask_lt();
        uint32_t n = c.pend_n;
#pragma unroll
        for (int j = 0; j < kUnroll; j++) {
            const uint32_t m = __ballot_sync(0xffffffffu, near[j]);
            if (near[j]) g_pend[warp_in_cta()][n + __popc(m & lt)] = v[j];
            n += __popc(m);
        }
        c.pend_n = n;
        if (n >= kPendT) drain_pending(a, c);
        return;
    }
#endif
#pragma unroll
    for (int j = 0; j < kUnroll; j++) any_near |= near[j];
    if (__any_sync(0xffffffffu, any_near)) {
        uint32_t cls[kUnroll];
#pragma unroll
        for (int j = 0; j < kUnroll; j++) cls[j] = near[j] ? class_of(a, v[j]) : 0u;
        push_near(a, near, v, cls, c);
    }
}

// Expand the out-arcs of up to 32 small vertices (one per lane) edge-balanced
// across the warp, kUnroll batches of 32 arcs at a time.
// skip (may be NULL): a lane whose vertex has its bit set there is dropped (the
// word is loaded together with the vertex's distance and row bounds).
template <typename OffT, bool UNIT>
__device__ __forceinline__ void expand_group(const GraphArgs<OffT> &a, bool valid, int32_t u, SweepCtx &c,
                                             const uint32_t *skip = nullptr) {
    uint32_t du = 0, deg = 0;
    OffT beg = 0;
    if (valid) {
        const uint32_t sk = skip ? __ldcg(skip + (u >> 5)) : 0u;
        du = __ldcg(a.dist + u);
        beg = __ldg(a.off + u);
        const OffT end = __ldg(a.off + u + 1);
        valid = ((sk >> (u & 31)) & 1u) == 0;
        deg = valid ? (uint32_t)(end - beg) : 0u;
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
        bool ok[kUnroll], ovf[kUnroll];
        int32_t v[kUnroll];
        uint32_t cand[kUnroll];
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
                v[j] = __ldcs(a.idx + e);
                w = UNIT ? 1u : __ldcs(a.w + e);
            }
            cand[j] = dq + w;
            ovf[j] = cand[j] < dq || cand[j] == kInf;
        }
        relax_multi(a, ok, v, cand, ovf, c);
    }
}

// Local chain: the warp pops up to 32 vertices at a time from the top of its
// stack (most recent first) and expands them, for at most g_sh.chain batches;
// whatever is left goes to the next sweep's worklist.  Warp-collective.
template <typename OffT, bool UNIT>
__device__ __forceinline__ void drain_local(const GraphArgs<OffT> &a, SweepCtx &c) {
    int32_t budget = g_sh.chain;
    while (c.lq_n > 0 && budget > 0) {
        __syncwarp();
        const uint32_t cnt = c.lq_n < 32u ? c.lq_n : 32u;
        const bool ok = lane_id() < cnt;
        const int32_t u = ok ? g_lq[warp_in_cta()][c.lq_n - cnt + lane_id()] : 0;
        __syncwarp();
        c.lq_n -= cnt;
        budget--;
        expand_group<OffT, UNIT>(a, ok, u, c);
    }
    if (c.lq_n > 0) {
        c.chain_on = false;
        while (c.lq_n > 0) {
            __syncwarp();
            const uint32_t cnt = c.lq_n < 32u ? c.lq_n : 32u;
            const bool w1[1] = {lane_id() < cnt};
            const int32_t u1[1] = {w1[0] ? g_lq[warp_in_cta()][c.lq_n - cnt + lane_id()] : 0};
            const uint32_t c1[1] = {w1[0] ? 1u : 0u};
            __syncwarp();
            c.lq_n -= cnt;
            push_near(a, w1, u1, c1, c);
        }
        c.chain_on = true;
    }
}

// One chunk (<= chunk_edges arcs) of one large vertex u: chunk y of the row
// [b0, e0), relaxed from d(u) = du.  Warp-collective; the arguments are
// warp-uniform.
template <typename OffT, bool UNIT>
__device__ __forceinline__ void chunk_body(const GraphArgs<OffT> &a, int32_t y, uint32_t du, OffT b0, OffT e0,
                                           SweepCtx &c) {
    const OffT size = (y & kFineFlag) ? (OffT)kFineChunk : (OffT)g_sh.chunk_edges;
    const int32_t yy = y & ~kFineFlag;
    const OffT beg = b0 + (OffT)yy * size;
    const OffT end = min(e0, beg + size);
    c.items += (lane_id() == 0 && yy == 0);
    c.edges += (lane_id() == 0) ? (uint32_t)(end - beg) : 0u;
    for (OffT base = beg; base < end; base += 32 * kUnroll) {
        bool ok[kUnroll], ovf[kUnroll];
        int32_t v[kUnroll];
        uint32_t cand[kUnroll];
#pragma unroll
        for (int j = 0; j < kUnroll; j++) {
            const OffT e = base + 32 * j + lane_id();
            ok[j] = e < end;
            v[j] = 0;
            uint32_t w = 0;
            if (ok[j]) {
                v[j] = __ldcs(a.idx + e);
                w = UNIT ? 1u : __ldcs(a.w + e);
            }
            cand[j] = du + w;
            ovf[j] = cand[j] < du || cand[j] == kInf;
        }
        relax_multi(a, ok, v, cand, ovf, c);
    }
}

// One chunk item (vertex u, chunk y): skipped when u was advanced again during
// this sweep (sweep k+1 expands it with the newer distance); the first chunk of
// a vertex clears its bit in B_k.  Warp-collective.
template <typename OffT, bool UNIT>
__device__ __forceinline__ void expand_chunk(const GraphArgs<OffT> &a, int2 item, SweepCtx &c) {
    const int32_t u = item.x;
    const uint32_t bit = 1u << (u & 31);
    uint32_t nxt = 0, du = 0;
    OffT b0 = 0, e0 = 0;
    if (lane_id() == 0) {
        nxt = __ldcg(g_sh.bm_next + (u >> 5));
        du = __ldcg(a.dist + u);
        b0 = __ldg(a.off + u);
        e0 = __ldg(a.off + u + 1);
        if ((item.y & ~kFineFlag) == 0) red_and(g_sh.bm_cur + (u >> 5), ~bit);
    }
    nxt = __shfl_sync(0xffffffffu, nxt, 0);
    if (nxt & bit) return;  // warp-uniform
    du = __shfl_sync(0xffffffffu, du, 0);
    b0 = __shfl_sync(0xffffffffu, b0, 0);
    e0 = __shfl_sync(0xffffffffu, e0, 0);
    chunk_body<OffT, UNIT>(a, item.y, du, b0, e0, c);
    if (c.chain_on) drain_local<OffT, UNIT>(a, c);
}

// Dense sweep item: g_sh.gw (<= kGroupWords) bitmap words (32 vertices each), loaded with
// one coalesced access.  The small vertices whose bit is set (and not set again
// for the next sweep) are compacted across the words, 32 per expansion, so a
// warp's lanes stay filled when few vertices of a word are active.  The words
// are cleared.
template <typename OffT, bool UNIT>
__device__ __forceinline__ void scan_words(const GraphArgs<OffT> &a, int64_t g, SweepCtx &c) {
    const int64_t w0 = g * g_sh.gw;
    const int64_t wi = w0 + lane_id();
    uint32_t act = 0;
    if (lane_id() < g_sh.gw && wi < a.nwords) {
        const uint32_t b = __ldcg(g_sh.bm_cur + wi);
        const uint32_t large = __ldg(&a.cls[wi].y);
        const uint32_t again = __ldcg(g_sh.bm_next + wi);
        if (b) {
            g_sh.bm_cur[wi] = 0u;
            act = b & ~large & ~again;
        }
    }
    const uint32_t cnt = __popc(act);
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < kGroupWords; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane_id() >= o) incl += t;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, kGroupWords - 1);
    const uint32_t excl = incl - cnt;
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t t = base + lane_id();
        int pos = 0;
#pragma unroll
        for (int sh = kGroupWords / 2; sh > 0; sh >>= 1) {
            const uint32_t probe = __shfl_sync(0xffffffffu, incl, pos + sh - 1);
            if (probe <= t) pos += sh;
        }
        const bool ok = t < total;
        const int owner = ok ? pos : 0;
        const uint32_t ex = __shfl_sync(0xffffffffu, excl, owner);
        const uint32_t word = __shfl_sync(0xffffffffu, act, owner);
        int32_t u = 0;
        if (ok) u = (int32_t)((w0 + owner) * 32 + __fns(word, 0, (int)(t - ex) + 1));
        expand_group<OffT, UNIT>(a, ok, u, c);
    }
}

// ---- pull sweeps (BFS over in-arcs; levels are exact per sweep, so the first
// in-neighbour found in the frontier B_k gives the least level k)
constexpr int kPullLaneRounds = 2;  // per-lane rounds of kPullUnroll in-arcs before the warp helps

// Up to 32 unreached vertices, one per lane (ok), v in bitmap word slot `owner`
// of the item.  Each lane scans its in-arcs kPullUnroll at a time and stops at
// the first source u with u in B_k; a vertex still open after
// kPullLaneRounds rounds is finished by the whole warp, 32 * kPullUnroll in-arcs
// per step.  A vertex found gets level d(u) + 1 and enters B_{k+1} (if it has
// out-arcs) and the worklists of sweep k+1.  Warp-collective.
template <typename OffT>
__device__ __forceinline__ void pull_batch(const GraphArgs<OffT> &a, bool ok, int32_t v, int owner, SweepCtx &c,
                                           uint32_t *s_found) {
    OffT b = 0, e = 0;
    if (ok) {
        b = __ldg(a.in_off + v);
        e = __ldg(a.in_off + v + 1);
    }
    c.items += ok;
    bool found = false;
    int32_t par = 0;
    uint32_t exam = 0;
#pragma unroll
    for (int r = 0; r < kPullLaneRounds; r++) {
        const bool act = ok && !found && b < e;
        if (!__any_sync(0xffffffffu, act)) break;
        int32_t u[kPullUnroll];
        bool in[kPullUnroll];
#pragma unroll
        for (int j = 0; j < kPullUnroll; j++) {
            in[j] = act && b + (OffT)j < e;
            u[j] = in[j] ? __ldg(a.in_idx + b + j) : 0;
        }
        uint32_t fw[kPullUnroll];
#pragma unroll
        for (int j = 0; j < kPullUnroll; j++) fw[j] = in[j] ? __ldcg(g_sh.bm_cur + (u[j] >> 5)) : 0u;
#pragma unroll
        for (int j = 0; j < kPullUnroll; j++) {
            if (in[j] && !found) {
                exam++;
                if ((fw[j] >> (u[j] & 31)) & 1u) {
                    found = true;
                    par = u[j];
                }
            }
        }
        if (act) b = (e - b > (OffT)kPullUnroll) ? b + (OffT)kPullUnroll : e;
    }
    uint32_t rest = __ballot_sync(0xffffffffu, ok && !found && b < e);
    while (rest) {
        const int l = __ffs(rest) - 1;
        rest &= rest - 1u;
        const OffT bl = __shfl_sync(0xffffffffu, b, l);
        const OffT el = __shfl_sync(0xffffffffu, e, l);
        int32_t hit = -1;
        uint32_t seen = 0;
        for (OffT base = bl; base < el && hit < 0; base += 32 * kPullUnroll) {
            int32_t u[kPullUnroll];
            bool in[kPullUnroll];
#pragma unroll
            for (int j = 0; j < kPullUnroll; j++) {
                const OffT x = base + (OffT)(32 * j + lane_id());
                in[j] = x < el;
                u[j] = in[j] ? __ldg(a.in_idx + x) : 0;
            }
            uint32_t fw[kPullUnroll];
#pragma unroll
            for (int j = 0; j < kPullUnroll; j++) fw[j] = in[j] ? __ldcg(g_sh.bm_cur + (u[j] >> 5)) : 0u;
#pragma unroll
            for (int j = 0; j < kPullUnroll; j++) {
                const uint32_t bal = __ballot_sync(0xffffffffu, in[j] && ((fw[j] >> (u[j] & 31)) & 1u));
                if (bal && hit < 0) hit = __shfl_sync(0xffffffffu, u[j], __ffs(bal) - 1);
            }
            seen += (uint32_t)min((OffT)(32 * kPullUnroll), el - base);
        }
        if (lane_id() == l) {
            exam += seen;
            if (hit >= 0) {
                found = true;
                par = hit;
            }
        }
    }
    c.edges += exam;
    uint32_t cls = 0;
    if (found) {
        const uint32_t dp = __ldcg(a.dist + par);
        cls = class_of(a, v);
        a.dist[v] = dp + 1u;
        atomicOr(&s_found[owner], 1u << (v & 31));
        c.adv++;
    }
    const bool nw[1] = {found && cls != 0};
    const int32_t vv[1] = {v};
    const uint32_t cc[1] = {cls};
    append_new(a, nw, vv, cc, c);
}

// Pull sweep item: kGroupWords bitmap words.  The vertices not reached yet
// (from the visited bitmap, or from their distances on the first pull sweep
// after push sweeps) are compacted 32 per batch; afterwards the item's words
// of the visited bitmap and of B_{k+1} are written whole (no other warp owns
// them in this sweep).
template <typename OffT>
__device__ __forceinline__ void pull_words(const GraphArgs<OffT> &a, int64_t g, SweepCtx &c, uint32_t *s_found) {
    const int64_t w0 = g * kGroupWords;
    const int q = lane_id();
    uint32_t unv = 0;  // lane q < kGroupWords: vertices of word w0 + q not reached yet
    if (g_sh.vis_valid) {
        if (q < kGroupWords && w0 + q < a.nwords) {
            unv = ~__ldcg(a.vis + w0 + q);
            const int64_t left = (int64_t)a.n - (w0 + q) * 32;
            if (left < 32) unv &= (1u << left) - 1u;
        }
    } else {
        uint32_t kv[kGroupWords];
#pragma unroll
        for (int j = 0; j < kGroupWords; j++) {
            const int64_t v = (w0 + j) * 32 + q;
            kv[j] = v < a.n ? __ldcg(a.dist + v) : 0u;
        }
#pragma unroll
        for (int j = 0; j < kGroupWords; j++) {
            const int64_t v = (w0 + j) * 32 + q;
            const uint32_t b = __ballot_sync(0xffffffffu, v < a.n && kv[j] == kInf);
            if (q == j) unv = b;
        }
    }
    if (q < kGroupWords) s_found[q] = 0u;
    __syncwarp();
    const uint32_t cnt = __popc(unv);
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < kGroupWords; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (q >= o) incl += t;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, kGroupWords - 1);
    const uint32_t excl = incl - cnt;
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t t = base + q;
        int pos = 0;
#pragma unroll
        for (int sh = kGroupWords / 2; sh > 0; sh >>= 1) {
            const uint32_t probe = __shfl_sync(0xffffffffu, incl, pos + sh - 1);
            if (probe <= t) pos += sh;
        }
        const bool ok = t < total;
        const int owner = ok ? pos : 0;
        const uint32_t ex = __shfl_sync(0xffffffffu, excl, owner);
        const uint32_t word = __shfl_sync(0xffffffffu, unv, owner);
        int32_t v = 0;
        if (ok) v = (int32_t)((w0 + owner) * 32 + __fns(word, 0, (int)(t - ex) + 1));
        pull_batch(a, ok, v, owner, c, s_found);
    }
    __syncwarp();
    if (q < kGroupWords && w0 + q < a.nwords) {
        const int64_t wi = w0 + q;
        const uint32_t f = s_found[q];
        if (!g_sh.vis_valid || f) a.vis[wi] = ~unv | f;
        const uint32_t nb = f & __ldg(&a.cls[wi].x);
        if (nb) g_sh.bm_next[wi] = nb;
    }
    __syncwarp();
}

// End of a sweep: the CTA publishes every warp's staged list entries with one
// reservation per list, and adds its dense_next mark count.
struct BlockFlush {
    uint32_t ns[16], nc[16];
    uint32_t base_s, base_c, marked;
    unsigned long long edges;        // arcs examined by the CTA in this sweep
    unsigned long long total_edges;  // ... in the run
    unsigned long long items, adv;   // run statistics of the CTA
};

template <typename OffT>
__device__ __forceinline__ void flush_sweep(const GraphArgs<OffT> &a, SweepCtx &c, BlockFlush *bf) {
    const int wid = threadIdx.x >> 5;
    const uint32_t nk = c.k + 1, nx = nk % 3;
    const uint32_t m = warp_sum(c.marked);
    c.marked = 0;
    const uint32_t de = warp_sum(c.edges);
    c.edges = 0;
    if (lane_id() == 0) {
        bf->ns[wid] = c.st_ns;
        bf->nc[wid] = c.st_nc;
        if (m) atomicAdd(&bf->marked, m);
        if (de) atomicAdd(&bf->edges, (unsigned long long)de);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t ts = 0, tc = 0;
        const int nw = blockDim.x >> 5;
        for (int i = 0; i < nw; i++) {
            const uint32_t xs = bf->ns[i], xc = bf->nc[i];
            bf->ns[i] = ts;
            bf->nc[i] = tc;
            ts += xs;
            tc += xc;
        }
        bf->base_s = (ts ? atomicAdd(&a.h->n_small[nx], ts) : 0u);
        bf->base_c = (tc ? atomicAdd(&a.h->n_chunk[nx], tc) : 0u);
        if (bf->marked) atomicAdd(&a.h->n_small[nx], bf->marked);
        bf->marked = 0;
        if (bf->edges) atomicAdd(&a.h->sweep_edges[c.k & 1], bf->edges);
        bf->total_edges += bf->edges;
        bf->edges = 0;
    }
    __syncthreads();
    int32_t *ls = pick2(a.small, nk) + bf->base_s + bf->ns[wid];
    for (uint32_t i = lane_id(); i < c.st_ns; i += 32) ls[i] = g_stage_small[warp_in_cta()][i];
    int2 *lc = pick2(a.chunk, nk) + bf->base_c + bf->nc[wid];
    for (uint32_t i = lane_id(); i < c.st_nc; i += 32) lc[i] = g_stage_chunk[warp_in_cta()][i];
    c.st_ns = 0;
    c.st_nc = 0;
}

// PULL: BFS with in-arcs (llp_bfs_pull); a separate instantiation keeps the
// pull code out of the register allocation of the push-only kernels.
template <typename OffT, bool UNIT, bool PULL>
__global__ void __launch_bounds__(512, LLP_SWEEP_MIN_BLOCKS) graph_sweep_kernel(GraphArgs<OffT> a) {
    __shared__ BlockFlush s_flush;
    __shared__ uint32_t s_work[2];
    __shared__ uint32_t s_cwork[2];
    WsHeader *h = a.h;
    const long long t0 = globaltimer_ns();
    const long long deadline = t0 + a.deadline_ns;
    uint32_t phase = 0;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
    const int warps_per_block = blockDim.x >> 5;
    const int64_t gwarp = (int64_t)blockIdx.x * warps_per_block + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * warps_per_block;
#ifdef LLP_SWEEP_TRACE
    __shared__ uint32_t s_first[2];
    if (threadIdx.x == 0) s_first[1] = 0xFFFFFFFFu;
#endif
    if (threadIdx.x == 0) {
        s_flush.marked = 0;
        s_flush.edges = 0;
        s_flush.total_edges = 0;
        s_flush.items = 0;
        s_flush.adv = 0;
        s_work[0] = 0;
        s_work[1] = 0;
        s_cwork[0] = 0;
        s_cwork[1] = 0;
    }

    SweepCtx c;
    // the schedule of this run: from the arguments, or chosen on the device (learned)
    int32_t small_max;
    {
        const bool dev = a.use_dev_sched && *(volatile int32_t *)&h->sched_valid;
        int32_t mode = a.mode, cfg = a.cfg, gw = a.group_words;
        uint32_t delta = a.delta;
        if (dev) {
            mode = *(volatile int32_t *)&h->sched_mode;
            delta = *(volatile uint32_t *)&h->sched_delta;
            cfg = *(volatile int32_t *)&h->sched_cfg;
            gw = *(volatile int32_t *)&h->sched_gw;
            if (mode < 0 || mode > 2) mode = LLP_MODE_AUTO;
            if (cfg < 1 || cfg > LLP_BLOCK_CFGS) cfg = 2;
            if (UNIT) delta = kInf;
        }
        const BlockCfg bcfg = block_cfg_of(cfg);
        small_max = bcfg.small_max;
        if (threadIdx.x == 0) {
            // dense items: the widest group that still gives every warp about three items
            if (gw != 1 && gw != 2 && gw != 4 && gw != kGroupWords) {
                const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
                gw = kGroupWords;
                while (gw > 1 && (int64_t)a.nwords / gw < 3 * warps) gw >>= 1;
            }
            g_sh.mode = mode;
            g_sh.cfg = cfg;
            g_sh.delta = delta;
            g_sh.small_max = bcfg.small_max;
            g_sh.chunk_edges = bcfg.chunk;
            g_sh.gw = gw;
            g_sh.chain = (dev ? *(volatile int32_t *)&h->sched_chain : a.local_chain);
            g_sh.fa = 0;
            g_sh.bucket_hi = (delta == kInf) ? (1ull << 40) : (unsigned long long)delta;
            g_sh.fixed_lo = 0;
            g_sh.pull = false;
            g_sh.vis_valid = false;
            g_sh.advance_bucket = false;
            g_sh.bm_next = a.bm[1];  // warm seeding appends to sweep 1
            if (!a.warm) {
                const uint32_t src_deg = (uint32_t)(__ldg(a.off + a.source + 1) - __ldg(a.off + a.source));
                const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
                g_sh.fine_src = src_deg > (uint32_t)bcfg.small_max &&
                                (int64_t)((src_deg + bcfg.chunk - 1) / bcfg.chunk) < warps;
            } else {
                g_sh.fine_src = false;
            }
        }
    }

    // ---- init_global_state / initial_states_to_process (paper Sec. 3.3)
    // a learned run had the state initialised by its prologue (for the default block
    // configuration); only the large bits change when the chosen one differs
    if (!a.pre_init) {
        const SweepInit<OffT> ini{a.n, a.source, a.warm, (uint32_t)small_max, a.off, a.dist, a.cls,
                                  a.bm[0], a.bm[1], a.bm[2], a.fixed};
        sweep_init(ini, gwarp, nwarps);
    } else if (small_max != a.small_max) {
        for (int64_t base = gwarp * 32; base < a.n; base += nwarps * 32) {
            const int64_t v = base + lane_id();
            const uint32_t deg = v < a.n ? (uint32_t)(__ldg(a.off + v + 1) - __ldg(a.off + v)) : 0u;
            const uint32_t large = __ballot_sync(0xffffffffu, deg > (uint32_t)small_max);
            if (lane_id() == 0) a.cls[base >> 5].y = large;
        }
    }
    if (gtid == 0) {
        h->t_start = t0;
        h->mode_used = g_sh.mode;
        h->delta_used = g_sh.delta;
        h->block_cfg_used = g_sh.cfg;
        for (int i = 0; i < 3; i++) h->far_min[i] = kInf;
        h->list_ok[1] = 1;
    }
    bool alive = grid_barrier(h, phase, deadline);
    if (a.warm && alive) {
        // initial_states_to_process of a warm start: every seed with a finite d and
        // out-arcs enters B_1 (deduplicated) and the worklists of sweep 1
        c.k = 0;
        for (int64_t base = gwarp * 32; base < a.n_seeds; base += nwarps * 32) {
            const int64_t i = base + lane_id();
            int32_t u = i < a.n_seeds ? a.seeds[i] : -1;
            if (i < a.n_seeds && (uint32_t)u >= (uint32_t)a.n) {
                set_status(h, LLP_ERR_INVALID_ARG);
                u = -1;
            }
            uint32_t cl = 0;
            bool nw = false;
            if (u >= 0) {
                cl = class_of(a, u);
                if (cl != 0 && __ldcg(a.dist + u) != kInf) {
                    const uint32_t bit = 1u << (u & 31);
                    nw = (atomicOr(a.bm[1] + (u >> 5), bit) & bit) == 0;
                }
            }
            const bool nw1[1] = {nw};
            const int32_t u1[1] = {u < 0 ? 0 : u};
            const uint32_t c1[1] = {cl};
            append_new(a, nw1, u1, c1, c);
        }
        flush_sweep(a, c, &s_flush);
    }
    if (blockIdx.x == 0 && alive && !a.warm) {
        // initial_states_to_process: the source (CTA 0 writes its list entries)
        const uint32_t src_deg = (uint32_t)(__ldg(a.off + a.source + 1) - __ldg(a.off + a.source));
        if (src_deg > 0) {
            if (threadIdx.x == 0) a.bm[1][a.source >> 5] = 1u << (a.source & 31);
            if (src_deg <= (uint32_t)g_sh.small_max) {
                if (threadIdx.x == 0) {
                    a.small[1][0] = a.source;
                    h->n_small[1] = 1;
                }
            } else {
                const uint32_t csize = g_sh.fine_src ? (uint32_t)kFineChunk : (uint32_t)g_sh.chunk_edges;
                const uint32_t nch = (src_deg + csize - 1) / csize;
                const int32_t flag = g_sh.fine_src ? kFineFlag : 0;
                for (uint32_t q = threadIdx.x; q < nch; q += blockDim.x)
                    a.chunk[1][q] = make_int2(a.source, (int)q | flag);
                if (threadIdx.x == 0) h->n_chunk[1] = nch;
            }
        }
    }
    if (alive) alive = grid_barrier(h, phase, deadline);

    if (gtid == 0) h->scratch[8] = (uint32_t)g_sh.chain;
    c.k = 1;
    uint32_t dense_sweeps = 0, pull_sweeps = 0;
    while (alive) {
        const uint32_t k = c.k;
        // thread 0 sets up the sweep for the CTA: it reads the worklist sizes once (the
        // same header words read by every warp of the grid queue up at one L2 slice)
        if (threadIdx.x == 0) {
            if (g_sh.advance_bucket) {
                g_sh.fixed_lo = g_sh.bucket_hi;  // the bucket just emptied: everything below it is final
                g_sh.bucket_hi = g_sh.next_hi;
                g_sh.fa += 1;
                g_sh.advance_bucket = false;
            }
            g_sh.prev_pull = g_sh.pull;
            g_sh.vis_valid = g_sh.pull;  // push sweeps reach vertices without recording them in vis
            g_sh.bm_cur = pick3(a.bm, k);
            g_sh.bm_next = pick3(a.bm, k + 1);
            const uint32_t ns = ld_relaxed_u32(&h->n_small[k % 3]);
            const uint32_t nc = ld_relaxed_u32(&h->n_chunk[k % 3]);
            g_sh.ns = ns;
            g_sh.nc = nc;
            g_sh.dense = ld_relaxed_u32(&h->list_ok[k % 3]) == 0;
            {
                const uint64_t per_warp = (uint64_t)ns / (uint64_t)nwarps;
                uint32_t gs = 32;
                while (gs > kMinGroup && per_warp < gs) gs >>= 1;
                g_sh.gsz = gs;
            }
            const unsigned long long csize = (k == 1 && g_sh.fine_src) ? (unsigned long long)kFineChunk
                                                                       : (unsigned long long)g_sh.chunk_edges;
            const unsigned long long arcs = (unsigned long long)ns * (unsigned long long)g_sh.small_max / 2 +
                                            (unsigned long long)nc * csize;
            bool dn = g_sh.mode == LLP_MODE_DENSE || (g_sh.mode == LLP_MODE_AUTO && arcs > a.dense_arcs);
            if (ns + nc == 0) dn = false;
            const bool pl = PULL && UNIT && g_sh.chain == 0 && ns + nc > 0 && arcs > a.pull_arcs;
            g_sh.pull = pl;
            g_sh.dense_next = dn && !pl;  // a pull sweep appends every vertex it reaches
            if (ns + nc == 0) {
                g_sh.nf = ld_relaxed_u32(&h->n_far[g_sh.fa % 3]);
                g_sh.fmin = ld_relaxed_u32(&h->far_min[g_sh.fa % 3]);
            }
        }
        __syncthreads();
        const uint32_t ns = g_sh.ns;
        const uint32_t nc = g_sh.nc;
        const bool dense = g_sh.dense;
        if (g_sh.prev_pull) {
            // B_{k-1} was read, not consumed, by the pull sweep k-1; it becomes B_{k+2}
            uint32_t *spare = pick3(a.bm, k + 2);
            for (int64_t wi = gtid; wi < a.nwords; wi += gthreads) spare[wi] = 0u;
        }
        if (threadIdx.x == 0) {  // used after the next grid barrier
            s_work[(k + 1) & 1] = 0;
            s_cwork[(k + 1) & 1] = 0;
        }
        if (gtid == 0) {
            const uint32_t r = (k + 2) % 3;
            h->n_small[r] = 0;
            h->n_chunk[r] = 0;
            h->work[r] = 0;
            h->list_ok[r] = 0;
            h->list_ok[(k + 1) % 3] = g_sh.dense_next ? 0u : 1u;
            if (k - 1 < kSweepLogCap)
                sweep_log(h)[k - 1] = SweepRec{(uint32_t)(globaltimer_ns() - t0), ns, nc,
                                               (dense ? 1u : 0u) | (ns + nc == 0 ? 2u : 0u)};
            // arcs examined by the previous sweep, in units of 1024 (bits 2..31 of its flags)
            const unsigned long long pe = *(volatile unsigned long long *)&h->sweep_edges[(k - 1) & 1];
            h->sweep_edges[(k - 1) & 1] = 0;
            if (k >= 2 && k - 2 < kSweepLogCap) {
                const unsigned long long q = min(pe >> 10, 0x3FFFFFFFull);
                sweep_log(h)[k - 2].flags |= (uint32_t)(q << 2);
            }
        }
        if (ns + nc == 0) {
            // near worklist empty: move to the next non-empty bucket, or stop
            const uint32_t nf = min(g_sh.nf, a.far_cap);
            if (nf == 0) break;
            const unsigned long long fmin = g_sh.fmin;
            const unsigned long long dl = g_sh.delta;
            unsigned long long nh = (fmin / dl + 1ull) * dl;
            if (nh < g_sh.bucket_hi + dl) nh = g_sh.bucket_hi + dl;
            if (gtid == 0) {
                h->n_far[(g_sh.fa + 2) % 3] = 0;
                h->far_min[(g_sh.fa + 2) % 3] = kInf;
                h->aux += 1;
            }
            const int2 *fl = pick2(a.far, g_sh.fa);
            for (int64_t base = gwarp * 32; base < nf; base += nwarps * 32) {
                const int64_t i = base + lane_id();
                const bool ok = i < nf;
                int2 e = make_int2(0, 0);
                bool live = false;
                if (ok) {
                    e = fl[i];
                    live = __ldcg(a.dist + e.x) == (uint32_t)e.y;
                }
                bool to_near[1] = {live && (unsigned long long)(uint32_t)e.y < nh};
                const bool keep = live && !to_near[0];
                const uint32_t slot = warp_append_slot(keep, &h->n_far[(g_sh.fa + 1) % 3]);
                if (keep) {
                    if (slot < a.far_cap) {
                        pick2(a.far, g_sh.fa + 1)[slot] = e;
                        atomicMin(&h->far_min[(g_sh.fa + 1) % 3], (uint32_t)e.y);
                    } else {
                        to_near[0] = true;
                    }
                }
                const int32_t vv[1] = {e.x};
                const uint32_t cl[1] = {ok ? class_of(a, e.x) : 0u};
                push_near(a, to_near, vv, cl, c);
            }
            if (threadIdx.x == 0) {  // taken at the start of the next sweep
                g_sh.next_hi = nh;
                g_sh.advance_bucket = true;
            }
        } else if (PULL && g_sh.pull) {
            pull_sweeps++;
            const uint32_t ngroups = (uint32_t)(((int64_t)a.nwords + kGroupWords - 1) / kGroupWords);
            uint32_t *s_found = reinterpret_cast<uint32_t *>(g_lq[warp_in_cta()]);  // no local chain in pull runs
            for (;;) {
                uint32_t j = 0;
                if (lane_id() == 0) j = atomicAdd(&s_work[k & 1], 1u);
                j = __shfl_sync(0xffffffffu, j, 0);
                const uint64_t g64 = (uint64_t)blockIdx.x + (uint64_t)j * gridDim.x;
                if (g64 >= ngroups) break;
                pull_words(a, (int64_t)g64, c, s_found);
            }
        } else {
            dense_sweeps += dense;
            // chunks: CTA b owns items b, b + G, b + 2G, ... (G = grid size; a hub's chunks
            // are consecutive in the list, so they spread over CTAs) and its warps take them
            // in turn from a shared counter (costs vary: skipped, partial and full chunks)
            const int2 *cl = pick2(a.chunk, k);
            c.chain_on = g_sh.chain > 0;
            // With many chunk items per warp (most of them skipped in the early sweeps of a
            // power-law graph) a warp takes kTake of its CTA's items at once and loads their
            // entries and "advanced again" words in parallel, one per lane; the survivors
            // are expanded in order (and tested again, as every chunk item is).
            const uint32_t take = (kTake > 1 && (uint64_t)nc >= (uint64_t)kTakeMin * nwarps) ? kTake : 1u;
            auto chunk_loop = [&]() {
                for (;;) {
                    uint32_t j = 0;
                    if (lane_id() == 0) j = atomicAdd(&s_cwork[k & 1], take);
                    j = __shfl_sync(0xffffffffu, j, 0);
                    if (take == 1) {
                        const uint64_t it = (uint64_t)blockIdx.x + (uint64_t)j * gridDim.x;
                        if (it >= nc) break;
                        expand_chunk<OffT, UNIT>(a, cl[it], c);
                        continue;
                    }
                    const uint64_t it = (uint64_t)blockIdx.x + (uint64_t)(j + lane_id()) * gridDim.x;
                    const bool ok = lane_id() < take && it < nc;
                    if (!__any_sync(0xffffffffu, ok)) break;
                    int2 item = make_int2(0, 0);
                    bool live = false;
                    if (ok) {
                        item = cl[it];
                        const uint32_t bit = 1u << (item.x & 31);
                        live = (__ldcg(g_sh.bm_next + (item.x >> 5)) & bit) == 0u;
                        if ((item.y & ~kFineFlag) == 0) red_and(g_sh.bm_cur + (item.x >> 5), ~bit);
                    }
                    uint32_t todo = __ballot_sync(0xffffffffu, live);
                    while (todo) {
                        const int q = __ffs(todo) - 1;
                        todo &= todo - 1u;
                        const int2 iq = make_int2(__shfl_sync(0xffffffffu, item.x, q), __shfl_sync(0xffffffffu, item.y, q));
                        expand_chunk<OffT, UNIT>(a, iq, c);
                    }
                }
            };
            // vertex groups (their cost varies): CTA b owns groups b, b + G, b + 2G, ...
            // (G = grid size) and its warps take them in turn from a shared counter
            auto group_loop = [&]() {
                const uint32_t gsz = g_sh.gsz;
                const uint32_t ngroups = dense ? (uint32_t)(((int64_t)a.nwords + g_sh.gw - 1) / g_sh.gw)
                                               : (uint32_t)(((uint64_t)ns + gsz - 1) / gsz);
                const int32_t *sl = pick2(a.small, k);
                for (;;) {
                    uint32_t j = 0;
                    if (lane_id() == 0) j = atomicAdd(&s_work[k & 1], 1u);
                    j = __shfl_sync(0xffffffffu, j, 0);
                    const uint64_t g64 = (uint64_t)blockIdx.x + (uint64_t)j * gridDim.x;
                    if (g64 >= ngroups) break;
                    const uint32_t g = (uint32_t)g64;
                    if (dense) {
                        scan_words<OffT, UNIT>(a, g, c);
                        if (c.chain_on) drain_local<OffT, UNIT>(a, c);
                    } else {
                        const int64_t i = (int64_t)g * gsz + lane_id();
                        bool ok = (uint32_t)lane_id() < gsz && i < ns;
                        int32_t u = ok ? sl[i] : 0;
                        if (ok) red_and(g_sh.bm_cur + (u >> 5), ~(1u << (u & 31)));
                        expand_group<OffT, UNIT>(a, ok, u, c, g_sh.bm_next);  // advanced again: next sweep
                        if (c.chain_on) drain_local<OffT, UNIT>(a, c);
                    }
                }
            };
            chunk_loop();
            group_loop();
#if LLP_DEFER
            if (c.pend_n) drain_pending(a, c);
#endif
            c.chain_on = false;
        }
#ifdef LLP_SWEEP_TRACE
        // s_first[k & 1] was reset during sweep k - 1 (a grid barrier separates the two)
        if (threadIdx.x == 0) s_first[(k + 1) & 1] = 0xFFFFFFFFu;
        if (lane_id() == 0) atomicMin(&s_first[k & 1], (uint32_t)(globaltimer_ns() - t0));
#endif
        flush_sweep(a, c, &s_flush);
#ifdef LLP_SWEEP_TRACE
        if (threadIdx.x == 0 && k - 1 < 64 && blockIdx.x < 1024) {
            a.trace[((k - 1) * 1024 + blockIdx.x) * 2] = s_first[k & 1];
            a.trace[((k - 1) * 1024 + blockIdx.x) * 2 + 1] = (uint32_t)(globaltimer_ns() - t0);
        }
#endif
        alive = grid_barrier(h, phase, deadline);
        c.k += 1;
    }

    // ---- final_solution: dist[] already holds G

    // ---- statistics (one atomic per CTA and counter)
    const uint32_t it_s = warp_sum(c.items), ad_s = warp_sum(c.adv);
    if (lane_id() == 0) {
        atomicAdd(&s_flush.items, (unsigned long long)it_s);
        atomicAdd(&s_flush.adv, (unsigned long long)ad_s);
    }
    if (gtid == 0) {
        h->sweeps = (int32_t)c.k;
        h->dense_sweeps = (int32_t)dense_sweeps;
        h->scratch[7] = pull_sweeps;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&h->items, s_flush.items);
        atomicAdd(&h->edges, s_flush.total_edges);
        atomicAdd(&h->advances, s_flush.adv);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t done = atomicAdd(&h->scratch[0], 1u) + 1u;
        if (done == gridDim.x) h->t_end = globaltimer_ns();
    }
}

struct Layout {
    uint2 *cls;
    uint32_t *bm[3];
    uint32_t *vis;
    uint32_t *fixed;
    int32_t *small[2];
    int2 *chunk[2];
    int2 *far[2];
    uint32_t far_cap;
    uint32_t *trace;
    void *lb_lists;  // the load-balanced engine's lists (they overlay the lists above)
    size_t bytes;
};

Layout carve_graph(void *ws, int32_t n, int64_t m) {
    Carve c(ws);
    Layout L;
    const size_t nwords = ((size_t)n + 31) / 32;
    // chunks of one sweep: sum over large v of ceil(deg/chunk) <= m/128 + m/17
    const size_t chunk_cap = (size_t)(m / 128 + m / 16 + 2);
    L.far_cap = (uint32_t)std::max<int64_t>(n, 1024);
    L.cls = c.take<uint2>(nwords);
    L.bm[0] = c.take<uint32_t>(nwords);
    L.bm[1] = c.take<uint32_t>(nwords);
    L.bm[2] = c.take<uint32_t>(nwords);
    L.vis = c.take<uint32_t>(nwords);
    L.fixed = c.take<uint32_t>(nwords);
    const size_t lists_at = c.off;
    L.small[0] = c.take<int32_t>(n);
    L.small[1] = c.take<int32_t>(n);
    L.chunk[0] = c.take<int2>(chunk_cap);
    L.chunk[1] = c.take<int2>(chunk_cap);
    L.far[0] = c.take<int2>(L.far_cap);
    L.far[1] = c.take<int2>(L.far_cap);
    // the load-balanced engine's lists overlay the lists above (one engine per call)
    const size_t lists_at_al = align_up(lists_at, 256);
    L.lb_lists = ws ? (void *)((char *)ws + lists_at_al) : nullptr;
    c.off = std::max(c.off, lists_at_al + lb_workspace_bytes(n, m));
#ifdef LLP_SWEEP_TRACE
    L.trace = c.take<uint32_t>(64 * 1024 * 2);
#else
    L.trace = nullptr;
#endif
    L.bytes = c.bytes();
    return L;
}

// Heuristic schedule (the fallback of the learned scheduler).
void resolve_schedule(const llp_sched_t *s, bool unit, int32_t n, int64_t m, int32_t &mode, uint32_t &delta,
                      int32_t &cfg, unsigned long long &dense_arcs, int &threads) {
    mode = s ? s->mode : LLP_MODE_AUTO;
    if (mode < 0 || mode > 2) mode = LLP_MODE_AUTO;
    delta = s ? s->delta : 0u;
    if (delta == 0u) delta = kInf;  // heuristic: one worklist
    if (unit) delta = kInf;         // unit weights: sweeps are BFS levels already
    cfg = s ? s->block_cfg : 0;
    if (cfg < 1 || cfg > LLP_BLOCK_CFGS) cfg = 2;
    // dense sweeps once a sweep touches more than permille/1000 of the arcs
    const int pm = (s && s->dense_permille > 0) ? s->dense_permille : 50;
    dense_arcs = (unsigned long long)m * (unsigned long long)pm / 1000ull;
    (void)n;
    threads = (s && (s->threads == 256 || s->threads == 512)) ? s->threads : 512;
}

template <bool UNIT>
llp_status_t graph_solve(const llp_csr_t *g, int32_t source, uint32_t *out, const llp_sched_t *s, void *ws,
                         size_t ws_bytes, cudaStream_t stream, const llp_csr_t *gin = nullptr,
                         const int32_t *seeds = nullptr, int32_t n_seeds = -1) {
    if (!g || !out || !ws) return LLP_ERR_INVALID_ARG;
    if (n_seeds > 0 && !seeds) return LLP_ERR_INVALID_ARG;
    if (gin && (gin->n != g->n || gin->m != g->m || gin->offsets_64 != g->offsets_64 || !gin->offsets ||
                (gin->m > 0 && !gin->indices)))
        return LLP_ERR_INVALID_ARG;
    if (g->n < 1 || g->n > (1 << 29) || g->m < 0 || !g->offsets) return LLP_ERR_INVALID_ARG;
    if (g->m > 0 && (!g->indices || (!UNIT && !g->weights))) return LLP_ERR_INVALID_ARG;
    if (!g->offsets_64 && g->m > 0x7FFFFFFFll) return LLP_ERR_INVALID_ARG;
    if (source < 0 || source >= g->n) return LLP_ERR_INVALID_ARG;
    if (((uintptr_t)ws & 255u) != 0) return LLP_ERR_INVALID_ARG;
    Layout L = carve_graph(ws, g->n, g->m);
    if (ws_bytes < L.bytes) return LLP_ERR_WORKSPACE_TOO_SMALL;

    int32_t mode, cfg;
    uint32_t delta;
    unsigned long long dense_arcs;
    int threads;
    resolve_schedule(s, UNIT, g->n, g->m, mode, delta, cfg, dense_arcs, threads);
    const BlockCfg bc = block_cfg_of(cfg);
    llp_status_t rc = reset_header(ws, stream);
    if (rc != LLP_OK) return rc;
    const bool learned = s && s->use_mlp && s->mlp_params;
    // pull sweeps: frontiers above m * permille / 1000 out-arcs (estimated as in AUTO mode)
    const int ppm = s ? s->pull_permille : 0;
    const bool pull_on = UNIT && gin && ppm >= 0;
    const unsigned long long pull_arcs = (unsigned long long)g->m * (unsigned long long)(ppm > 0 ? ppm : 200) / 1000ull;

    // Block configuration 4 selects the load-balanced engine (lb_sweep.cu): one worklist (no
    // buckets), no local chain, no pull sweeps, the schedule chosen on the host, int32 offsets.
    const int lchain = (s && s->local_chain > 0) ? s->local_chain : 0;
    const bool lb_ok = s && s->block_cfg == 4 && !learned && !pull_on && !g->offsets_64 && delta == kInf &&
                       lchain == 0;
    if (lb_ok) {
        return lb_launch(UNIT, g, source, out, L.bm[0], L.bm[1], L.lb_lists, (WsHeader *)ws, deadline_from(s), mode,
                         dense_arcs, seeds, n_seeds, stream);
    }
    // Grid size: small graphs sweep faster on fewer CTAs (their sweeps are short chains of
    // dependent loads plus a grid barrier whose cost grows with the CTA count); one CTA per
    // 1,024 vertices, at least 32, at most every co-resident CTA.
    const int max_blocks = (int)std::max<int64_t>(32, ((int64_t)g->n + 1023) / 1024);
    auto fill = [&](auto &args) {
        args.n = g->n;
        args.source = source;
        args.idx = g->indices;
        args.w = UNIT ? nullptr : g->weights;
        args.dist = out;
        args.nwords = (int32_t)(((int64_t)g->n + 31) / 32);
        args.cls = L.cls;
        args.bm[0] = L.bm[0];
        args.bm[1] = L.bm[1];
        args.bm[2] = L.bm[2];
        args.vis = L.vis;
        args.in_idx = pull_on ? gin->indices : nullptr;
        args.pull_arcs = pull_arcs;
        args.small[0] = L.small[0];
        args.small[1] = L.small[1];
        args.chunk[0] = L.chunk[0];
        args.chunk[1] = L.chunk[1];
        args.far[0] = L.far[0];
        args.far[1] = L.far[1];
        args.far_cap = L.far_cap;
        args.trace = L.trace;
        args.fixed = (!UNIT && s && s->fixed_memo > 0 && delta != kInf) ? L.fixed : nullptr;
        args.h = (WsHeader *)ws;
        args.delta = delta;
        args.mode = mode;
        args.dense_arcs = dense_arcs;
        args.small_max = bc.small_max;
        args.chunk_edges = bc.chunk;
        args.cfg = cfg;
        args.use_dev_sched = learned ? 1 : 0;
        args.pre_init = learned ? 1 : 0;
        args.local_chain = (s && s->local_chain > 0) ? s->local_chain : 0;
        args.group_words = s ? s->group_words : 0;
        args.deadline_ns = deadline_from(s);
        args.warm = n_seeds >= 0 ? 1 : 0;
        args.n_seeds = n_seeds > 0 ? n_seeds : 0;
        args.seeds = seeds;
    };
    // a learned run: one prologue launch computes the schedule (features + network) while its
    // other CTAs initialise the state for the default block configuration
    auto prologue = [&](const auto &args) -> llp_status_t {
        using OffT = std::remove_cv_t<std::remove_pointer_t<decltype(args.off)>>;
        const SweepInit<OffT> ini{args.n, args.source, args.warm, (uint32_t)args.small_max, args.off, args.dist,
                                  args.cls, args.bm[0], args.bm[1], args.bm[2], args.fixed};
        return enqueue_learned_prologue<OffT>(g, source, UNIT, s->mlp_params, (WsHeader *)ws, ini, stream);
    };
    if (g->offsets_64) {
        GraphArgs<int64_t> args;
        fill(args);
        args.off = (const int64_t *)g->offsets;
        if (learned) {
            rc = prologue(args);
            if (rc != LLP_OK) return rc;
        }
        args.in_off = pull_on ? (const int64_t *)gin->offsets : nullptr;
        void *kargs[] = {&args};
        const void *fn = (const void *)graph_sweep_kernel<int64_t, UNIT, false>;
        if constexpr (UNIT) {
            if (pull_on) fn = (const void *)graph_sweep_kernel<int64_t, true, true>;
        }
        return launch_cooperative(fn, threads, 0, max_blocks, kargs, stream);
    } else {
        GraphArgs<int32_t> args;
        fill(args);
        args.off = (const int32_t *)g->offsets;
        if (learned) {
            rc = prologue(args);
            if (rc != LLP_OK) return rc;
        }
        args.in_off = pull_on ? (const int32_t *)gin->offsets : nullptr;
        void *kargs[] = {&args};
        const void *fn = (const void *)graph_sweep_kernel<int32_t, UNIT, false>;
        if constexpr (UNIT) {
            if (pull_on) fn = (const void *)graph_sweep_kernel<int32_t, true, true>;
        }
        return launch_cooperative(fn, threads, 0, max_blocks, kargs, stream);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Scratch for llp_sssp_noalloc: a fixed device array owned by this library.
// It exists once per GPU that loads the library and stays allocated until the
// process exits.  Host code must not pass `g_noalloc_scratch` itself to a
// kernel (on the host that name is only a stand-in for the symbol); the device
// address is looked up with cudaGetSymbolAddress, once per device.
constexpr size_t kNoallocScratchBytes = (size_t)64 << 20;  // 64 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64];  // device address of the scratch, per device ordinal

// Returns the device address of the scratch array on the current device,
// looking it up on first use (must not happen during stream capture).
llp_status_t noalloc_scratch(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        (void)cudaGetLastError();
        return LLP_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return LLP_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return LLP_OK;
}

}  // namespace
}  // namespace llp

extern "C" {

size_t llp_sssp_noalloc_max_workspace(void) { return llp::kNoallocScratchBytes; }

llp_status_t llp_sssp_noalloc(const llp_csr_t *g, int32_t source, uint32_t *dist, const llp_sched_t *sched,
                              void *stream) {
    if (!g || g->n < 1 || g->m < 0) return LLP_ERR_INVALID_ARG;
    const size_t need = llp::carve_graph(nullptr, g->n, g->m).bytes;
    if (need > llp::kNoallocScratchBytes) return LLP_ERR_WORKSPACE_TOO_SMALL;
    void *scratch = nullptr;
    const llp_status_t rc = llp::noalloc_scratch(&scratch);
    if (rc != LLP_OK) return rc;
    return llp::graph_solve<false>(g, source, dist, sched, scratch, llp::kNoallocScratchBytes,
                                   (cudaStream_t)stream);
}

llp_status_t llp_sssp_noalloc_status(int32_t *status, void *stream) {
    if (!status) return LLP_ERR_INVALID_ARG;
    void *scratch = nullptr;
    const llp_status_t rc = llp::noalloc_scratch(&scratch);
    if (rc != LLP_OK) return rc;
    // the status word is the first field of the header at the start of the scratch
    int32_t st = 0;
    LLP_CUDA_TRY(cudaMemcpyAsync(&st, scratch, sizeof(st), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    LLP_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    *status = st;
    return LLP_OK;
}

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

llp_status_t llp_sssp_warm(const llp_csr_t *g, int32_t source, uint32_t *dist, const int32_t *seeds, int32_t n_seeds,
                           const llp_sched_t *sched, void *ws, size_t ws_bytes, void *stream) {
    if (n_seeds < 0) return LLP_ERR_INVALID_ARG;
    return llp::graph_solve<false>(g, source, dist, sched, ws, ws_bytes, (cudaStream_t)stream, nullptr, seeds,
                                   n_seeds);
}

llp_status_t llp_bfs_warm(const llp_csr_t *g, int32_t source, uint32_t *level, const int32_t *seeds, int32_t n_seeds,
                          const llp_sched_t *sched, void *ws, size_t ws_bytes, void *stream) {
    if (n_seeds < 0) return LLP_ERR_INVALID_ARG;
    return llp::graph_solve<true>(g, source, level, sched, ws, ws_bytes, (cudaStream_t)stream, nullptr, seeds,
                                  n_seeds);
}

llp_status_t llp_bfs_pull(const llp_csr_t *g, const llp_csr_t *g_in, int32_t source, uint32_t *level,
                          const llp_sched_t *sched, void *ws, size_t ws_bytes, void *stream) {
    if (!g_in) return LLP_ERR_INVALID_ARG;
    return llp::graph_solve<true>(g, source, level, sched, ws, ws_bytes, (cudaStream_t)stream, g_in);
}

}  // extern "C"

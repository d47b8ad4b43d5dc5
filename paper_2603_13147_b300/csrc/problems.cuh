// CTA-level LLP solvers shared by the single-instance entry points and the
// batched engine.  Each routine solves one whole instance with the threads of
// one CTA, sweeps separated by __syncthreads (a CTA-local barrier).
#pragma once

#include "llp_common.cuh"

namespace llp {

constexpr unsigned long long kEmptySuitor = 0xFFFFFFFFFFFFFFFFull;

// 64-bit atomic min with acquire-release ordering at device scope (generic
// address: global or shared memory); returns the previous value.
__device__ __forceinline__ unsigned long long atomic_min_acq_rel(unsigned long long *p, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.acq_rel.gpu.min.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

// ------------------------------------------------------------ stable marriage
// Paper Sec. 4.3.  G[m] = next[m], the index into man m's list.  m is
// forbidden iff the woman w he targets holds a suitor she ranks better; the
// predicate is evaluated in O(1) against best[w] = packed (rank << 32 | man)
// minimum over every man that ever targeted w (the all-time best suitor is the
// only one never forbidden at w, so "ever" equals "currently").  Advance moves m
// to his next choice.  A thread carries one free man; when its man displaces
// another, it continues with the displaced one (his advance follows at once),
// so no sweep barrier is needed.  Returns the number of proposals.
// `best` may live in shared or global memory (generic pointer); `next` too.
__device__ __forceinline__ unsigned long long propose_chain(int32_t m, int32_t k, int32_t n, const int32_t *men_pref,
                                                            const int32_t *women_rank,
                                                            unsigned long long *best, int32_t *next,
                                                            WsHeader *h, long long deadline, bool &failed) {
    constexpr int L = 8;  // look-ahead: the next L women of m are checked with independent loads
    unsigned long long proposals = 0, rounds = 0;
    for (;;) {
        if (k >= n) {  // list exhausted: Algorithm LLP's "null" (advance beyond T[m])
            set_status(h, LLP_ERR_INFEASIBLE);
            failed = true;
            return proposals;
        }
        if ((++rounds & 255ull) == 0 && globaltimer_ns() > deadline) {
            set_status(h, LLP_ERR_TIMEOUT);
            failed = true;
            return proposals;
        }
        const int32_t cnt = (n - k) < L ? (n - k) : L;
        const int32_t *pr = men_pref + (int64_t)m * n + k;
        int32_t w[L];
        unsigned long long mine[L], cur[L];
#pragma unroll
        for (int i = 0; i < L; i++) w[i] = i < cnt ? __ldg(pr + i) : 0;
#pragma unroll
        for (int i = 0; i < L; i++)
            mine[i] = i < cnt ? (((unsigned long long)(uint32_t)__ldg(women_rank + (int64_t)w[i] * n + m) << 32) |
                                 (uint32_t)m)
                              : 0ull;
#pragma unroll
        for (int i = 0; i < L; i++) cur[i] = i < cnt ? *(volatile unsigned long long *)(best + w[i]) : 0ull;
        // forbidden at w[i] (w already holds a better suitor) for every i before the first candidate
        int cand = -1;
#pragma unroll
        for (int i = L - 1; i >= 0; i--)
            if (i < cnt && cur[i] > mine[i]) cand = i;
        if (cand < 0) {
            proposals += cnt;
            k += cnt;
            continue;
        }
        proposals += cand + 1;
        k += cand;
        unsigned long long my = 0;
        int32_t ww = 0;
#pragma unroll
        for (int i = 0; i < L; i++)
            if (i == cand) {
                my = mine[i];
                ww = w[i];
            }
        next[m] = k;
        // acq_rel: the release orders next[m] before m becomes w's suitor; the acquire makes
        // the displaced man's next[] (stored before his own proposal) visible below
        const unsigned long long old = atomic_min_acq_rel(best + ww, my);
        if (old < my) {  // lost the race: forbidden after all
            k++;
            continue;
        }
        if (old == kEmptySuitor) return proposals;  // w was free: chain ends
        // m displaced old's man, who is forbidden now: carry him
        m = (int32_t)(uint32_t)(old & 0xFFFFFFFFull);
        k = *(volatile int32_t *)(next + m) + 1;
    }
}

// ------------------------------------------------------------------ knapsack
// Paper Sec. 4.7.  Row `row` (W+1 int32 cells, shared or global memory) holds
// G[k-1, *] before item k and G[k, *] after it.  Capacities are processed top
// down in chunks of blockDim.x * R cells: every cell of a chunk computes
// max(G[k-1,c], v_k + G[k-1,c-w_k]) into registers, the CTA synchronises, then
// writes; cells below the chunk are still G[k-1, *] when read, so one buffer
// suffices.  Items with w < 1 or v < 0 set LLP_ERR_INVALID_ARG in h.
// One item over capacities [wk, top), top-down chunks, in place.
template <int R>
__device__ __forceinline__ void knapsack_item(int32_t wk, int32_t vk, int32_t top, int32_t *row) {
    const int32_t T = blockDim.x;
    const int32_t tid = threadIdx.x;
    const int32_t chunk = T * R;
    for (; top - chunk >= wk; top -= chunk) {
        const int32_t *src = row + (top - chunk) + tid;
        int32_t nv[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int32_t keep = src[r * T];
            const int32_t take = src[r * T - wk] + vk;
            nv[r] = keep > take ? keep : take;
        }
        __syncthreads();
        int32_t *dst = row + (top - chunk) + tid;
#pragma unroll
        for (int r = 0; r < R; r++) dst[r * T] = nv[r];
    }
    if (top > wk) {
        int32_t nv[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int32_t c = wk + r * T + tid;
            nv[r] = 0;
            if (c < top) {
                const int32_t keep = row[c];
                const int32_t take = row[c - wk] + vk;
                nv[r] = keep > take ? keep : take;
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int32_t c = wk + r * T + tid;
            if (c < top) row[c] = nv[r];
        }
    }
}

template <int R>
__device__ __forceinline__ void knapsack_cta(int32_t n, const int32_t *w, const int32_t *v, int32_t W, int32_t *row,
                                             WsHeader *h) {
    const int32_t T = blockDim.x;
    const int32_t tid = threadIdx.x;
    for (int32_t c = tid; c <= W; c += T) row[c] = 0;
    __syncthreads();
    const int32_t chunk = T * R;  // capacities are < 2^26, so 32-bit indices suffice
    int32_t k = 0;
    while (k < n) {
        const int32_t wa = __ldg(w + k), va = __ldg(v + k);
        if (wa < 1 || va < 0) {  // outside the problem statement: report, skip
            if (tid == 0 && h) set_status(h, LLP_ERR_INVALID_ARG);
            k++;
            continue;
        }
        const int32_t wb = k + 1 < n ? __ldg(w + k + 1) : 0, vb = k + 1 < n ? __ldg(v + k + 1) : 0;
        if (k + 1 < n && wb >= 1 && vb >= 0 && (int64_t)wa + wb <= W) {
            // Two items (a, b) per pass for the capacities c >= w_a + w_b: the new
            // row is max(n1[c], n1[c - w_b] + v_b) with n1[x] = max(o[x], o[x - w_a] + v_a),
            // which reads the previous row o at c, c - w_a, c - w_b, c - w_a - w_b,
            // all at or below c, so the top-down in-place chunking stays valid.
            // 4 loads + 1 store per two cell updates instead of 6 + 2, half the barriers.
            const int32_t wab = wa + wb;
            int32_t top = W + 1;
            for (; top - chunk >= wab; top -= chunk) {
                const int32_t *src = row + (top - chunk) + tid;
                int32_t nv[R];
#pragma unroll
                for (int r = 0; r < R; r++) {
                    const int32_t oc = src[r * T];
                    const int32_t oa = src[r * T - wa];
                    const int32_t ob = src[r * T - wb];
                    const int32_t oab = src[r * T - wab];
                    const int32_t n1c = oc > oa + va ? oc : oa + va;
                    const int32_t n1b = ob > oab + va ? ob : oab + va;
                    nv[r] = n1c > n1b + vb ? n1c : n1b + vb;
                }
                __syncthreads();
                int32_t *dst = row + (top - chunk) + tid;
#pragma unroll
                for (int r = 0; r < R; r++) dst[r * T] = nv[r];
            }
            __syncthreads();
            // the capacities below: item a then item b, one at a time
            const int32_t lo_top = top;  // cells [lo_top, W] hold both items already
            knapsack_item<R>(wa, va, lo_top, row);
            __syncthreads();
            // item b over [wb, lo_top): cells in [lo_top, lo_top + wb) read only below lo_top... but
            // cells >= lo_top are final, so b must only touch [wb, lo_top)
            knapsack_item<R>(wb, vb, lo_top, row);
            __syncthreads();
            k += 2;
            continue;
        }
        if (wa <= W) knapsack_item<R>(wa, va, W + 1, row);
        __syncthreads();
        k++;
    }
}

// Sum of values (int64) by the CTA; used to reject instances whose optimum can
// overflow int32 before sweeping.
__device__ __forceinline__ long long cta_sum_i32(int32_t n, const int32_t *v) {
    __shared__ long long s_part[32];
    long long acc = 0;
    for (int32_t i = threadIdx.x; i < n; i += blockDim.x) acc += __ldg(v + i);
    acc = warp_sum(acc);
    if (lane_id() == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    long long tot = 0;
    if (threadIdx.x < 32) {
        tot = (threadIdx.x < (blockDim.x >> 5)) ? s_part[threadIdx.x] : 0;
        tot = warp_sum(tot);
        if (threadIdx.x == 0) s_part[0] = tot;
    }
    __syncthreads();
    tot = s_part[0];
    __syncthreads();
    return tot;
}

}  // namespace llp

namespace llp {

// ------------------------------------------------------------ job scheduling
// Paper Sec. 4.4 on one CTA.  off[0..n] are the job rows' arc positions (in
// the caller's concatenated successor array), idx[] local successor ids in
// [0, n).  maxp/remaining/list0/list1 are CTA-private (shared or global).
// Level-synchronous: a job enters the worklist when its last predecessor is
// fixed, is advanced to maxp + t and fixed, and publishes to its successors.
// Returns the number of fixed jobs (< n means a cycle).
__device__ __forceinline__ int32_t job_cta(int32_t n, const int64_t *off, const int32_t *idx, const int32_t *dur,
                                           int32_t *completion, int32_t *maxp, int32_t *remaining, int32_t *list0,
                                           int32_t *list1, WsHeader *h) {
    __shared__ int32_t s_cnt[2];
    __shared__ int32_t s_fixed;
    const int T = blockDim.x;
    for (int32_t j = threadIdx.x; j < n; j += T) {
        maxp[j] = 0;
        remaining[j] = 0;
    }
    if (threadIdx.x == 0) {
        s_cnt[0] = 0;
        s_cnt[1] = 0;
        s_fixed = 0;
    }
    __syncthreads();
    const int64_t e0 = off[0], e1 = off[n];
    for (int64_t e = e0 + threadIdx.x; e < e1; e += T) {
        const int32_t s = __ldg(idx + e);
        if ((uint32_t)s < (uint32_t)n) atomicAdd(remaining + s, 1);
        else set_status(h, LLP_ERR_INVALID_ARG);
    }
    __syncthreads();
    for (int32_t j = threadIdx.x; j < n; j += T)
        if (remaining[j] == 0) list0[atomicAdd(&s_cnt[0], 1)] = j;
    __syncthreads();
    int cur = 0;
    int32_t fixed_local = 0;
    for (;;) {
        const int32_t cnt = s_cnt[cur];
        if (cnt == 0) break;
        const int32_t *L = cur ? list1 : list0;
        int32_t *N = cur ? list0 : list1;
        for (int32_t i = threadIdx.x; i < cnt; i += T) {
            const int32_t j = L[i];
            long long c = (long long)maxp[j] + __ldg(dur + j);
            if (c > 0x7FFFFFFFll) {
                set_status(h, LLP_ERR_OVERFLOW);
                c = 0x7FFFFFFF;
            }
            completion[j] = (int32_t)c;
            fixed_local++;
            for (int64_t e = off[j]; e < off[j + 1]; e++) {
                const int32_t s = __ldg(idx + e);
                atomicMax(maxp + s, (int32_t)c);
                if (atomicSub(remaining + s, 1) == 1) N[atomicAdd(&s_cnt[cur ^ 1], 1)] = s;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_cnt[cur] = 0;
        cur ^= 1;
        __syncthreads();
    }
    atomicAdd(&s_fixed, fixed_local);
    __syncthreads();
    const int32_t fixed = s_fixed;
    __syncthreads();
    return fixed;
}

// ------------------------------------------------------------ small SSSP / BFS
// Paper Sec. 4.1 / 4.2 on one CTA.  d[] (n uint32, the state G) and the
// frontier bitmaps cur/nxt (ceil(n/32) words each) are CTA-private: shared
// memory, or global memory for large n (d may then be the output itself).
// Sweep k expands the vertices whose bit is set in cur (advanced in sweep
// k-1): warps take bitmap words in turn and expand a word's set vertices
// together, their arcs balanced across the lanes; a candidate d(u) + w(u,v)
// below d(v) makes v forbidden, the advance is an atomic min on d[v] and v's
// bit is set in nxt.  A word of cur is cleared as it is read, so cur is empty
// when it becomes nxt.  The CTA barrier ends a sweep; the run stops after a
// sweep that advanced nothing.  off[] are the rows' arc positions in the
// caller's concatenated arrays, idx[] local target ids.  Returns the number of
// sweeps; arcs += arcs examined (per thread).
__device__ __forceinline__ int32_t graph_cta(int32_t n, const int64_t *off, const int32_t *idx, const uint32_t *w,
                                             bool unit, int32_t src, uint32_t *d, uint32_t *cur, uint32_t *nxt,
                                             WsHeader *h, long long deadline, unsigned long long &arcs) {
    constexpr int U = 4;  // arcs per lane in flight
    __shared__ int s_more[3];
    __shared__ int s_stop;
    const int32_t nwords = (n + 31) >> 5;
    const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int32_t v = threadIdx.x; v < n; v += blockDim.x) d[v] = 0xFFFFFFFFu;
    for (int32_t i = threadIdx.x; i < nwords; i += blockDim.x) {
        cur[i] = 0u;
        nxt[i] = 0u;
    }
    if (threadIdx.x == 0) {
        s_more[0] = 1;
        s_stop = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        d[src] = 0u;
        cur[src >> 5] = 1u << (src & 31);
    }
    __syncthreads();
    int32_t k = 0;
    for (;;) {
        k++;
        if (threadIdx.x == 0) {
            s_more[k % 3] = 0;
            if (globaltimer_ns() > deadline) {
                set_status(h, LLP_ERR_TIMEOUT);
                s_stop = 1;
            }
        }
        __syncthreads();
        if (s_stop) break;
        bool more = false;
        for (int32_t wi = warp; wi < nwords; wi += nwarp) {
            const uint32_t bits = *(volatile uint32_t *)&cur[wi];
            if (bits == 0u) continue;
            __syncwarp();
            if (lane == 0) cur[wi] = 0u;
            const bool own = lane < __popc(bits);
            const int32_t u = own ? (wi << 5) + (int32_t)__fns(bits, 0, lane + 1) : 0;
            uint32_t du = 0, deg = 0;
            int64_t beg = 0;
            if (own) {
                du = *(volatile uint32_t *)&d[u];
                beg = off[u];
                deg = (uint32_t)(off[u + 1] - beg);
            }
            uint32_t incl = deg;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            const uint32_t excl = incl - deg;
            arcs += (lane == 0) ? total : 0u;
            for (uint32_t base = 0; base < total; base += 32 * U) {
                int32_t v[U];
                uint64_t cand[U];
                bool ok[U];
#pragma unroll
                for (int j = 0; j < U; j++) {
                    const uint32_t t = base + 32 * j + lane;
                    int pos = 0;
#pragma unroll
                    for (int sh = 16; sh > 0; sh >>= 1) {
                        const uint32_t probe = __shfl_sync(0xffffffffu, incl, pos + sh - 1);
                        if (probe <= t) pos += sh;
                    }
                    ok[j] = t < total;
                    const int owner = ok[j] ? pos : 0;
                    const uint32_t ex = __shfl_sync(0xffffffffu, excl, owner);
                    const int64_t bo = __shfl_sync(0xffffffffu, beg, owner);
                    const uint32_t dq = __shfl_sync(0xffffffffu, du, owner);
                    v[j] = 0;
                    uint32_t wt = 0;
                    if (ok[j]) {
                        const int64_t e = bo + (int64_t)(t - ex);
                        v[j] = __ldg(idx + e);
                        wt = unit ? 1u : __ldg(w + e);
                    }
                    cand[j] = (uint64_t)dq + wt;
                }
#pragma unroll
                for (int j = 0; j < U; j++) {
                    if (!ok[j]) continue;
                    if (cand[j] >= 0xFFFFFFFFull) {
                        set_status(h, LLP_ERR_OVERFLOW);
                        s_stop = 1;
                    } else if ((uint32_t)cand[j] < *(volatile uint32_t *)&d[v[j]]) {
                        atomicMin(&d[v[j]], (uint32_t)cand[j]);
                        atomicOr(&nxt[v[j] >> 5], 1u << (v[j] & 31));
                        more = true;
                    }
                }
            }
        }
        if (more) s_more[k % 3] = 1;
        __syncthreads();
        if (!s_more[k % 3] || s_stop) break;
        uint32_t *t = cur;
        cur = nxt;
        nxt = t;
    }
    return k;
}

// ------------------------------------------------------- stable marriage CTA
// Paper Sec. 4.3 on one CTA: best[] and next[] CTA-private (shared memory for
// n <= a few thousand).  Threads take men in turn and carry displacement
// chains to their end (propose_chain).  Writes wife[m].  Returns proposals.
__device__ __forceinline__ unsigned long long marriage_cta(int32_t n, const int32_t *men_pref,
                                                           const int32_t *women_rank, int32_t *wife,
                                                           unsigned long long *best, int32_t *next, WsHeader *h,
                                                           long long deadline) {
    for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
        best[i] = kEmptySuitor;
        next[i] = 0;
    }
    __syncthreads();
    unsigned long long props = 0;
    bool failed = false;
    for (int32_t m = threadIdx.x; m < n && !failed; m += blockDim.x)
        props += propose_chain(m, 0, n, men_pref, women_rank, best, next, h, deadline, failed);
    __syncthreads();
    for (int32_t m = threadIdx.x; m < n; m += blockDim.x) {
        const int32_t k = next[m];
        wife[m] = (k >= 0 && k < n) ? __ldg(men_pref + (int64_t)m * n + k) : -1;
    }
    __syncthreads();
    return props;
}

}  // namespace llp

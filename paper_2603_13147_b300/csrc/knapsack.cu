// 0-1 knapsack as an LLP (paper Sec. 4.7), single instance.
//
// Cell G[k,c] = best value of items 0..k-1 within capacity c; G[0,*] = 0 is
// the bottom.  A cell is forbidden while it is below
// max(G[k-1,c], v_k + G[k-1,c-w_k]); the advance raises it to that bound.  Row
// k depends only on row k-1, so one CTA sweeps the capacity range once per
// item with the recurrence evaluated for every cell in parallel and a CTA
// barrier between items (knapsack_cta).  The row lives in shared memory when
// it fits (W+1 <= 56K cells), otherwise in the workspace (L1/L2 resident).
//
// Large single instances run as a wavefront over capacity slices instead
// (knapsack_wave, below): one CTA per slice on every SM, no grid-wide barrier
// per item; a CTA waits only for the cells of lower slices it reads.
//
// The thread-block cluster kernel (knapsack_cluster, opt-in with block
// configuration 3): CTA r of a cluster of CL CTAs (one per SM) owns capacities
// [r*S, (r+1)*S) of the row, double-buffered in its shared memory; a cell's
// lower neighbours G[k-1, c - w] that another CTA owns are read from that CTA's
// shared memory (distributed shared memory), and one cluster barrier separates
// passes.  Each pass applies K items at once: G[k+K-1, c] = max over the
// subsets T of the K items that fit of G[k-1, c - w(T)] + v(T) (the recurrence
// unrolled K times, all terms read from the row before the pass), so the
// dependent chain of barriers is n/K long (K = 2 measured fastest).
#include <algorithm>
#include <cooperative_groups.h>

#include "llp_common.cuh"
#include "problems.cuh"

namespace cg = cooperative_groups;

namespace llp {
namespace {

constexpr int kKnapThreads = 1024;
constexpr int kKnapR = 8;
constexpr int32_t kSmemCells = 56 * 1024;  // 224 KB of int32

__global__ void __launch_bounds__(kKnapThreads) knapsack_single(int32_t n, const int32_t *w, const int32_t *v,
                                                               int32_t W, int32_t *best, int32_t *final_row,
                                                               int32_t *grow, WsHeader *h) {
    extern __shared__ int32_t srow[];
    const long long t0 = globaltimer_ns();
    if (cta_sum_i32(n, v) > 0x7FFFFFFFll) {
        if (threadIdx.x == 0) set_status(h, LLP_ERR_OVERFLOW);
        return;
    }
    int32_t *row = (W + 1 <= kSmemCells) ? srow : grow;
    knapsack_cta<kKnapR>(n, w, v, W, row, h);
    if (final_row)
        for (int32_t c = threadIdx.x; c <= W; c += blockDim.x) final_row[c] = row[c];
    if (threadIdx.x == 0) {
        best[0] = row[W];
        h->t_start = t0;
        h->t_end = globaltimer_ns();
        h->sweeps = n;
        h->items = (unsigned long long)n;
        h->edges = (unsigned long long)n * (unsigned long long)(W + 1);
    }
}

constexpr int kClusterThreads = 1024;
#ifndef LLP_KNAP_CLUSTER_K
#define LLP_KNAP_CLUSTER_K 2
#endif
constexpr int kClusterK = LLP_KNAP_CLUSTER_K;  // items per pass
constexpr int kClusterCells = 4;    // cells per thread in flight

// Address of the int32 at shared-memory offset `a` (bytes, this CTA's window) in
// the shared memory of cluster CTA `rank`, and a load from it.
__device__ __forceinline__ uint32_t cluster_addr(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
// The rows read in a pass do not change during it (cluster barriers separate the
// passes), so the loads are left free to be scheduled together.
__device__ __forceinline__ int32_t ld_cluster(uint32_t addr) {
    int32_t v;
    asm("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

// One instance on one cluster of gridDim.x CTAs; S cells of the row per CTA (a
// multiple of 1024), two buffers of S int32 in dynamic shared memory.  inv_s =
// floor(2^32 / S) + 1 gives x / S with one correction step.
template <int K>
__global__ void __launch_bounds__(kClusterThreads) knapsack_cluster(int32_t n, const int32_t *w, const int32_t *v,
                                                                    int32_t W, int32_t S, uint32_t inv_s,
                                                                    int32_t *best, int32_t *final_row, WsHeader *h) {
    extern __shared__ int32_t sbuf[];
    cg::cluster_group cluster = cg::this_cluster();
    const int32_t rank = (int32_t)cluster.block_rank();
    const int32_t T = blockDim.x, tid = threadIdx.x;
    const long long t0 = globaltimer_ns();
    const bool over = cta_sum_i32(n, v) > 0x7FFFFFFFll;  // every CTA computes it: same answer
    if (over) {
        if (rank == 0 && tid == 0) set_status(h, LLP_ERR_OVERFLOW);
        return;
    }
    const int32_t lo = rank * S;
    for (int32_t i = tid; i < S; i += T) sbuf[i] = 0;  // G[0, *] = 0 (buffer 0)
    cluster.sync();
    constexpr int NS = 1 << K;
    int32_t pass = 0;
    for (int32_t k = 0; k < n; k += K, pass++) {
        // subset sums of items k .. k+K-1 (an invalid or missing item never fits)
        int32_t ws[NS], vs[NS];
        int32_t wi[K], vi[K];
#pragma unroll
        for (int j = 0; j < K; j++) {
            wi[j] = W + 1;
            vi[j] = 0;
            if (k + j < n) {
                const int32_t a = __ldg(w + k + j), b = __ldg(v + k + j);
                if (a < 1 || b < 0) {
                    if (rank == 0 && tid == 0) set_status(h, LLP_ERR_INVALID_ARG);
                } else {
                    wi[j] = a > W ? W + 1 : a;
                    vi[j] = b;
                }
            }
        }
#pragma unroll
        for (int m = 0; m < NS; m++) {
            long long sw = 0;
            int32_t sv = 0;
#pragma unroll
            for (int j = 0; j < K; j++)
                if (m & (1 << j)) {
                    sw += wi[j];
                    sv += vi[j];
                }
            ws[m] = sw > W ? W + 1 : (int32_t)sw;
            vs[m] = sv;
        }
        const int32_t *src = sbuf + (pass & 1) * S;
        int32_t *dst = sbuf + ((pass + 1) & 1) * S;
        const uint32_t src_sh = (uint32_t)__cvta_generic_to_shared(src);
        for (int32_t i0 = 0; i0 < S; i0 += T * kClusterCells) {
            int32_t b[kClusterCells];
#pragma unroll
            for (int q = 0; q < kClusterCells; q++) {
                const int32_t c = lo + i0 + q * T + tid;
                const bool live = i0 + q * T + tid < S && c <= W;
                // every term is loaded (a term that does not fit reads the cell itself and is
                // dropped below), so all the loads of a cell group can be in flight together
                const int32_t cc = live ? c : lo;
                int32_t val[NS];
#pragma unroll
                for (int m = 0; m < NS; m++) {
                    const bool fits = ws[m] <= cc;
                    const uint32_t x = (uint32_t)(fits ? cc - ws[m] : cc);
                    uint32_t r = __umulhi(x, inv_s);
                    if (r * (uint32_t)S > x) r--;
                    val[m] = ld_cluster(cluster_addr(src_sh + 4u * (x - r * (uint32_t)S), r)) + (fits ? vs[m] : 0);
                }
                b[q] = val[0];
#pragma unroll
                for (int m = 1; m < NS; m++) b[q] = b[q] > val[m] ? b[q] : val[m];
            }
#pragma unroll
            for (int q = 0; q < kClusterCells; q++) {
                const int32_t i = i0 + q * T + tid;
                if (i < S) dst[i] = b[q];
            }
        }
        cluster.sync();
    }
    const int32_t *row = sbuf + (pass & 1) * S;
    if (final_row)
        for (int32_t i = tid; i < S && lo + i <= W; i += T) final_row[lo + i] = row[i];
    if (W >= lo && W < lo + S && tid == 0) best[0] = row[W - lo];
    if (rank == 0 && tid == 0) {
        h->t_start = t0;
        h->t_end = globaltimer_ns();
        h->sweeps = (n + K - 1) / K;
        h->items = (unsigned long long)n;
        h->edges = (unsigned long long)n * (unsigned long long)(W + 1);
    }
    cluster.sync();  // no CTA leaves while another may still read its row
}

// ---------------------------------------------------------------------------
// Wavefront over capacity slices (knapsack_wave): CTA s of P co-resident CTAs owns
// the capacities [s*S, (s+1)*S) and keeps its part of G[k] and G[k+1] in shared
// memory.  Row k+1 depends on row k at c and c - w_k, and c - w_k < c, so a CTA
// only ever waits for CTAs below it: no grid-wide barrier per item.  Every cell
// of G[k] is also written to a ring of R rows in global memory (L2-resident) as
// one 64-bit word, value | k << 32; a CTA that needs G[k][x] of a lower slice
// takes the ring word only when its tag is k (the data carry their own
// readiness: no fence, no flag on the dependency path) and loads the words of
// kWaveF items ahead of use.  Each CTA publishes the number of items it has done
// (relaxed store, per block of kWaveF items); before overwriting the ring slot of
// G[j], a CTA waits until every CTA that may read it (those within the largest
// item weight above it) has done item j.  Every wait is bounded by the call's
// deadline; a CTA that gives up raises the header's abort flag, which the others
// check while waiting.
#ifndef LLP_WAVE_T
#define LLP_WAVE_T 512
#endif
constexpr int kWaveThreads = LLP_WAVE_T;
#ifndef LLP_WAVE_F
#define LLP_WAVE_F 4
#endif
constexpr int kWaveF = LLP_WAVE_F;  // items per block (ring loads in flight, progress published per block)
constexpr int kWaveWin = 1024;
  // items whose parameters are staged in shared memory at a time

__device__ __forceinline__ unsigned long long ld_ring(const unsigned long long *p) {
    unsigned long long x;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(x) : "l"(p));
    return x;
}
// No "memory" clobber: the shared-memory work of the item may move across the store (the
// ring words carry their own tags; volatile asm keeps the ring and progress accesses in order,
// and the CTA barrier orders the shared row).
__device__ __forceinline__ void st_ring(unsigned long long *p, unsigned long long x) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(x));
}
__device__ __forceinline__ void st_relaxed_u32(uint32_t *p, uint32_t x) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(x) : "memory");
}

// Gives up a wait: timeout status and the abort flag (first caller), or a
// deadline check every 64 spins.  Returns true when the wait must end.
__device__ __forceinline__ bool wave_give_up(WsHeader *h, uint32_t spins, long long deadline) {
    if ((spins & 63u) != 63u) return false;
    if (ld_relaxed_u32(&h->abort_flag)) return true;
    if (globaltimer_ns() > deadline) {
        set_status(h, LLP_ERR_TIMEOUT);
        atomicExch(&h->abort_flag, 1u);
        return true;
    }
    return false;
}

template <int Q>
__global__ void __launch_bounds__(kWaveThreads, 1)
    knapsack_wave(int32_t n, const int32_t *w, const int32_t *v, int32_t W, int32_t S, int32_t R,
                  unsigned long long *ring, uint32_t *prog, int32_t *best, int32_t *final_row, WsHeader *h,
                  long long deadline_ns) {
    extern __shared__ int32_t sbuf[];
    __shared__ int2 s_item[kWaveWin];  // (weight, value) of the items of the current window
    __shared__ int s_abort;
    __shared__ int32_t s_wmax;
    __shared__ long long s_known;  // a lower bound of the readers' published item counts
    const int32_t s = blockIdx.x, P = gridDim.x, tid = threadIdx.x, T = blockDim.x;
    const long long t0 = globaltimer_ns();
    const long long deadline = t0 + deadline_ns;
    const int32_t lo = s * S, hi = min(lo + S, W + 1);
    const size_t row_len = (size_t)W + 1;
    if (cta_sum_i32(n, v) > 0x7FFFFFFFll) {  // every CTA computes it: same answer
        if (s == 0 && tid == 0) set_status(h, LLP_ERR_OVERFLOW);
        return;
    }
    // largest weight of an item that fits (its reads reach that far below a cell)
    if (tid == 0) {
        s_wmax = 0;
        s_abort = 0;
        s_known = 0;
    }
    __syncthreads();
    int32_t wm = 0;
    for (int32_t i = tid; i < n; i += T) {
        const int32_t a = __ldg(w + i);
        if (a <= W && a > wm) wm = a;
    }
    atomicMax(&s_wmax, wm);
    int32_t *prev = sbuf, *cur = sbuf + S;
    for (int32_t i = tid; i < S; i += T) prev[i] = 0;  // G[0] = 0
    // the CTAs that read this CTA's cells: those whose slice starts within s_wmax above it
    __syncthreads();
    const int32_t reach = min(P - 1, s + 1 + (s_wmax + S - 1) / S);
    // ring words of the lower slices for one block of items (ahead of use: the next block's
    // words are loaded while the current block runs)
    auto prefetch = [&](int32_t kb0, unsigned long long (&pf)[kWaveF][Q]) {
#pragma unroll
        for (int j = 0; j < kWaveF; j++) {
            const int32_t k = kb0 + j;
            const int32_t wj = k < n ? s_item[k % kWaveWin].x : W + 1;
#pragma unroll
            for (int q = 0; q < Q; q++) {
                const int32_t c = lo + tid + q * T;
                const int32_t x = c - wj;
                const bool rd = c < hi && wj <= c && x < lo && k >= 1;
                pf[j][q] = rd ? ld_ring(ring + (size_t)(k & (R - 1)) * row_len + x) : 0ull;
            }
        }
    };
    unsigned long long pf_cur[kWaveF][Q], pf_nxt[kWaveF][Q];
    for (int32_t k0 = 0; k0 < n; k0 += kWaveF) {
        const int32_t kb = min(kWaveF, n - k0);
        if (k0 % kWaveWin == 0) {
            // next window of item parameters (an item outside the problem statement never fits)
            __syncthreads();
            for (int32_t i = tid; i < kWaveWin && k0 + i < n; i += T) {
                int32_t a = __ldg(w + k0 + i), b = __ldg(v + k0 + i);
                if (a < 1 || b < 0) {
                    set_status(h, LLP_ERR_INVALID_ARG);
                    a = W + 1;
                    b = 0;
                }
                s_item[i] = make_int2(a > W ? W + 1 : a, b);
            }
            __syncthreads();
            prefetch(k0, pf_nxt);
        }
#pragma unroll
        for (int j = 0; j < kWaveF; j++)
#pragma unroll
            for (int q = 0; q < Q; q++) pf_cur[j][q] = pf_nxt[j][q];
        if ((k0 + kWaveF) % kWaveWin != 0 && k0 + kWaveF < n) prefetch(k0 + kWaveF, pf_nxt);
        // this block writes G[k0+1 .. k0+kb] over G[k0+1-R .. k0+kb-R]; a CTA reads G[j] during item j,
        // so every reader must have done items up to k0+kb-R (published count >= k0+kb-R+1)
        const int64_t need = (int64_t)k0 + kb - R + 1;
        if (need > s_known) {  // uniform: s_known changes only between CTA barriers
            __syncthreads();
            if (tid < 32) {
                for (uint32_t spins = 0;; spins++) {
                    uint32_t mn = 0xFFFFFFFFu;
                    for (int32_t c2 = s + 1 + tid; c2 <= reach; c2 += 32)
                        mn = min(mn, ld_relaxed_u32(prog + (size_t)c2 * 32));
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
                    if ((int64_t)mn >= need) {
                        if (tid == 0) s_known = (long long)mn;
                        break;
                    }
                    if (__any_sync(0xffffffffu, wave_give_up(h, spins, deadline))) {
                        if (tid == 0) s_abort = 1;
                        break;
                    }
                }
            }
            __syncthreads();  // no warp writes the block's ring rows before the readers are done
            if (s_abort) break;
        }
        bool quit = false;
#pragma unroll
        for (int j = 0; j < kWaveF; j++) {
            if (j >= kb) break;
            const int32_t k = k0 + j;
            const int2 it = s_item[k % kWaveWin];
            const int32_t wj = it.x, vj = it.y;
            unsigned long long *dst = ring + (size_t)((k + 1) & (R - 1)) * row_len;
#pragma unroll
            for (int q = 0; q < Q; q++) {
                const int32_t c = lo + tid + q * T;
                if (c < hi) {
                    int32_t g = prev[c - lo];
                    if (wj <= c) {
                        const int32_t x = c - wj;
                        int32_t lower;
                        if (x >= lo) {
                            lower = prev[x - lo];
                        } else if (k == 0) {
                            lower = 0;
                        } else {
                            unsigned long long e = pf_cur[j][q];
                            const unsigned long long *src = ring + (size_t)(k & (R - 1)) * row_len + x;
                            for (uint32_t spins = 0; (uint32_t)(e >> 32) != (uint32_t)k; spins++) {
                                if (wave_give_up(h, spins, deadline)) {
                                    s_abort = 1;
                                    break;
                                }
                                e = ld_ring(src);
                            }
                            lower = (int32_t)(uint32_t)e;
                        }
                        const int32_t cand = lower + vj;
                        g = cand > g ? cand : g;
                    }
                    cur[c - lo] = g;
                    st_ring(dst + c, ((unsigned long long)(uint32_t)(k + 1) << 32) | (uint32_t)g);
                }
            }
            __syncthreads();
            int32_t *t = prev;
            prev = cur;
            cur = t;
            if (s_abort) {
                quit = true;
                break;
            }
        }
        if (quit) break;
        if (tid == 0) st_relaxed_u32(prog + (size_t)s * 32, (uint32_t)(k0 + kb));
    }
    if (s_abort) return;
    if (final_row)
        for (int32_t c = lo + tid; c < hi; c += T) final_row[c] = prev[c - lo];
    if (W >= lo && W < hi && tid == 0) best[0] = prev[W - lo];
    if (s == 0 && tid == 0) {
        h->t_start = t0;
        h->t_end = globaltimer_ns();
        h->sweeps = n;
        h->items = (unsigned long long)n;
        h->edges = (unsigned long long)n * (unsigned long long)(W + 1);
    }
}

// Slices, cells per thread and ring rows of the wavefront for capacity W (cl = 0:
// W too large for Q <= 8 cells per thread on the co-resident CTAs).
struct WavePlan {
    int P = 0, Q = 0;
    int32_t S = 0, R = 0;
    size_t smem = 0;
};

#ifndef LLP_WAVE_Q
#define LLP_WAVE_Q 1
#endif
#ifndef LLP_WAVE_R
#define LLP_WAVE_R 256
#endif

WavePlan plan_wave(int32_t n, int32_t W) {
    WavePlan pl;
    const DeviceInfo di = device_info();
    if (di.sms <= 0) return pl;
    const int64_t cells = (int64_t)W + 1;
    // about LLP_WAVE_Q cells per thread; more only when the SMs run out
    int Q = LLP_WAVE_Q;
    int64_t P = (cells + (int64_t)kWaveThreads * Q - 1) / ((int64_t)kWaveThreads * Q);
    while (P > di.sms && Q < 8) {
        Q *= 2;
        P = (cells + (int64_t)kWaveThreads * Q - 1) / ((int64_t)kWaveThreads * Q);
    }
    if (P > di.sms || P < 2) return pl;
    pl.P = (int)P;
    pl.Q = Q;
    pl.S = (int32_t)((cells + P - 1) / P);
    // a power of two (slots by mask), at least two blocks and one row more, at most what the items need
    int32_t R = 1;
    while (R < 2 * kWaveF + 2 || (R < LLP_WAVE_R && R < n + 1)) R *= 2;
    pl.R = R;
    pl.smem = (size_t)pl.S * 2 * 4;
    return pl;
}

size_t wave_workspace_bytes(const WavePlan &pl, int32_t W) {
    if (pl.P == 0) return 0;
    return align_up((size_t)pl.R * ((size_t)W + 1) * 8, 256) + (size_t)pl.P * 128;
}

// Cluster size and cells per CTA for capacity W, or 0 when the row does not fit
// the cluster's shared memory (the single-CTA kernel then runs it).
struct ClusterPlan {
    int cl = 0;
    int32_t S = 0;
    uint32_t inv_s = 0;
    size_t smem = 0;
};

ClusterPlan plan_cluster(int32_t W) {
    ClusterPlan best;
    const DeviceInfo di = device_info();
    for (int cl : {16, 8}) {
        // S: a multiple of the CTA size, and the fewest CTAs (at most cl) that cover W + 1 cells
        const int64_t S = (((int64_t)W + 1 + cl - 1) / cl + kClusterThreads - 1) / kClusterThreads * kClusterThreads;
        const int ncta = (int)(((int64_t)W + 1 + S - 1) / S);
        const size_t smem = (size_t)S * 2 * 4;
        if (smem + 1024 > (size_t)di.max_smem_optin) continue;
        auto fn = knapsack_cluster<kClusterK>;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
            (cl > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
            (void)cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(ncta);
        cfg.blockDim = dim3(kClusterThreads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = ncta;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess || nclusters < 1) {
            (void)cudaGetLastError();
            continue;
        }
        best.cl = ncta;
        best.S = (int32_t)S;
        best.inv_s = (uint32_t)((1ull << 32) / (uint64_t)S + 1ull);
        best.smem = smem;
        return best;
    }
    return best;
}

}  // namespace
}  // namespace llp

extern "C" {

size_t llp_knapsack_workspace_size(int32_t n_items, int32_t capacity) {
    if (n_items < 0 || capacity < 0) return 0;
    size_t b = llp::kHeaderBytes;
    size_t extra = capacity + 1 > llp::kSmemCells ? llp::align_up((size_t)(capacity + 1) * 4, 256) : 0;
    extra = std::max(extra, llp::wave_workspace_bytes(llp::plan_wave(n_items, capacity), capacity));
    return b + extra;
}

llp_status_t llp_knapsack(int32_t n_items, const int32_t *w, const int32_t *v, int32_t capacity, int32_t *best,
                          int32_t *final_row, const llp_sched_t *sched, void *ws, size_t ws_bytes, void *stream) {
    using namespace llp;
    if (n_items < 0 || capacity < 0 || capacity > (1 << 26) || !best || !ws) return LLP_ERR_INVALID_ARG;
    if (n_items > 0 && (!w || !v)) return LLP_ERR_INVALID_ARG;
    if (((uintptr_t)ws & 255u) != 0) return LLP_ERR_INVALID_ARG;
    if (ws_bytes < llp_knapsack_workspace_size(n_items, capacity)) return LLP_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t st = (cudaStream_t)stream;
    llp_status_t rc = reset_header(ws, st);
    if (rc != LLP_OK) return rc;
    // instances with more than a few thousand cell updates per item take a cluster
    const bool big = (int64_t)n_items * (int64_t)(capacity + 1) >= (1ll << 22) && capacity >= 4096 &&
                     (!sched || sched->block_cfg != 1);
    const bool wave = big && (!sched || sched->block_cfg != 3);
    if (wave) {
        const WavePlan pl = plan_wave(n_items, capacity);
        if (pl.P > 0) {
            unsigned long long *ring = (unsigned long long *)((char *)ws + kHeaderBytes);
            const size_t ring_bytes = (size_t)pl.R * ((size_t)capacity + 1) * 8;
            uint32_t *prog = (uint32_t *)((char *)ws + kHeaderBytes + align_up(ring_bytes, 256));
            // tags 0 never match a row read (rows 1..n): stale words of an earlier call are cleared
            LLP_CUDA_TRY(cudaMemsetAsync(ring, 0, ring_bytes, st));
            LLP_CUDA_TRY(cudaMemsetAsync(prog, 0, (size_t)pl.P * 128, st));
            long long dl = deadline_from(sched);
            int32_t S = pl.S, R = pl.R;
            void *args[] = {&n_items, (void *)&w, (void *)&v, &capacity, &S, &R, &ring, &prog, &best, &final_row,
                            &ws, &dl};
            const void *fn = pl.Q == 1 ? (const void *)knapsack_wave<1>
                           : pl.Q == 2 ? (const void *)knapsack_wave<2>
                           : pl.Q == 4 ? (const void *)knapsack_wave<4> : (const void *)knapsack_wave<8>;
            if (pl.smem > 48 * 1024)
                LLP_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem));
            // the CTAs wait for one another: all P must be co-resident, else the cluster kernel runs it
            int per_sm = 0;
            LLP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kWaveThreads, pl.smem));
            if ((int64_t)per_sm * device_info().sms >= pl.P) {
                int grid = 0;
                rc = launch_cooperative(fn, kWaveThreads, pl.smem, pl.P, args, st, &grid);
                if (rc != LLP_OK) return rc;
                return grid == pl.P ? LLP_OK : LLP_ERR_CUDA;
            }
        }
    }
    if (big) {
        const ClusterPlan pl = plan_cluster(capacity);
        if (pl.cl > 0) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(pl.cl);
            cfg.blockDim = dim3(kClusterThreads);
            cfg.dynamicSmemBytes = pl.smem;
            cfg.stream = st;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = pl.cl;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            LLP_CUDA_TRY(cudaLaunchKernelEx(&cfg, knapsack_cluster<kClusterK>, n_items, w, v, capacity, pl.S, pl.inv_s, best,
                                            final_row, (WsHeader *)ws));
            return LLP_OK;
        }
    }
    const bool in_smem = capacity + 1 <= kSmemCells;
    const size_t smem = in_smem ? (size_t)(capacity + 1) * 4 : 0;
    if (smem > 48 * 1024)
        LLP_CUDA_TRY(cudaFuncSetAttribute(knapsack_single, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          kSmemCells * 4));
    int32_t *grow = in_smem ? nullptr : (int32_t *)((char *)ws + kHeaderBytes);
    knapsack_single<<<1, kKnapThreads, smem, st>>>(n_items, w, v, capacity, best, final_row, grow, (WsHeader *)ws);
    LLP_CUDA_TRY(cudaGetLastError());
    return LLP_OK;
}

}  // extern "C"

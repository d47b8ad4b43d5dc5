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
// Large single instances run on a thread-block cluster instead (knapsack_cluster):
// CTA r of a cluster of CL CTAs (one per SM) owns capacities [r*S, (r+1)*S) of
// the row, double-buffered in its shared memory; a cell's lower neighbours
// G[k-1, c - w] that another CTA owns are read from that CTA's shared memory
// (distributed shared memory), and one cluster barrier separates passes.  Each
// pass applies K items at once: G[k+K-1, c] = max over the subsets T of the K
// items that fit of G[k-1, c - w(T)] + v(T) (the recurrence unrolled K times,
// all terms read from the row before the pass), so the dependent chain of
// barriers is n/K long (K = 2: each pass costs about as many remote loads as
// cells x 2^K, so 2 items per pass measured fastest, 1 and 3 close behind).
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
    if (capacity + 1 > llp::kSmemCells) b += llp::align_up((size_t)(capacity + 1) * 4, 256);
    return b;
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

// Batched LLP engine: thousands of uneven instances of four problem families
// (0-1 knapsack, job scheduling, stable marriage, small SSSP/BFS) solved in ONE persistent
// launch.  Each CTA repeatedly takes the next instance from a global queue and
// solves it entirely on its own (the CTA-level solvers of problems.cuh: the
// sweeps of one instance are separated by __syncthreads instead of grid
// barriers, and the instance state lives in shared memory when it fits).
//
// The queue order is planned on the device by a one-CTA kernel: every instance
// gets a cost estimate (knapsack: cells n*(W+1); jobs: arcs and jobs; marriage:
// expected proposals n*ln n; graphs: vertices and arcs), and a counting sort on log2(cost) puts the most
// expensive first (longest-processing-time order), so the tail of the launch
// is made of small instances.  The launch shape (threads per CTA, knapsack
// register blocking) is picked by llp_batch_autotune, which times candidates.
#include <math.h>

#include <algorithm>

#include "llp_common.cuh"
#include "problems.cuh"

namespace llp {
namespace {

enum : uint32_t { kFamKnap = 0, kFamJob = 1, kFamSm = 2, kFamGraph = 3 };

struct BatchArgs {
    llp_batch_t b;
    uint32_t *order;      // planned queue: (family << 30) | instance
    uint32_t total;
    char *cta_scratch;    // per-CTA global scratch (instances too big for shared memory)
    size_t cta_scratch_bytes;
    size_t smem_bytes;    // dynamic shared memory per CTA
    WsHeader *h;
    long long deadline_ns;
};

__device__ __forceinline__ uint32_t cost_bucket(double cost) {
    if (cost < 1.0) return 0;
    const int e = ilogb(cost);
    return (uint32_t)min(max(e, 0), 63);
}

// One CTA: cost buckets, histogram, descending prefix, scatter.
__global__ void __launch_bounds__(1024) batch_plan_kernel(BatchArgs a) {
    __shared__ uint32_t hist[64];
    __shared__ uint32_t base[64];
    const llp_batch_t &b = a.b;
    if (threadIdx.x < 64) hist[threadIdx.x] = 0;
    __syncthreads();
    auto cost_of = [&](uint32_t i, uint32_t &fam, uint32_t &inst) -> double {
        if (i < (uint32_t)b.knap_count) {
            fam = kFamKnap;
            inst = i;
            const double n = (double)(b.knap_item_off[i + 1] - b.knap_item_off[i]);
            return n * ((double)b.knap_capacity[i] + 1.0);
        }
        i -= b.knap_count;
        if (i < (uint32_t)b.job_count) {
            fam = kFamJob;
            inst = i;
            const int64_t j0 = b.job_off[i], j1 = b.job_off[i + 1];
            const double m = (double)(b.job_succ_offsets[j1] - b.job_succ_offsets[j0]);
            return 64.0 * ((double)(j1 - j0) + m);
        }
        i -= b.job_count;
        if (i < (uint32_t)b.sm_count) {
            fam = kFamSm;
            inst = i;
            const double n = (double)b.sm_n[i];
            return 256.0 * n * (log(n + 1.0) + 1.0);
        }
        i -= b.sm_count;
        fam = kFamGraph;
        inst = i;
        const int64_t v0 = b.gr_off[i], v1 = b.gr_off[i + 1];
        const double m = (double)(b.gr_arc_offsets[v1] - b.gr_arc_offsets[v0]);
        return 128.0 * ((double)(v1 - v0) + m);
    };
    for (uint32_t i = threadIdx.x; i < a.total; i += blockDim.x) {
        uint32_t f, x;
        atomicAdd(&hist[cost_bucket(cost_of(i, f, x))], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int k = 63; k >= 0; k--) {  // most expensive bucket first
            base[k] = run;
            run += hist[k];
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < a.total; i += blockDim.x) {
        uint32_t f, x;
        const uint32_t k = cost_bucket(cost_of(i, f, x));
        a.order[atomicAdd(&base[k], 1u)] = (f << 30) | x;
    }
}

template <int R>
__global__ void __launch_bounds__(1024, 1) batch_solve_kernel(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_item;
    WsHeader *h = a.h;
    const llp_batch_t &b = a.b;
    const long long t0 = globaltimer_ns();
    const long long deadline = t0 + a.deadline_ns;
    if (blockIdx.x == 0 && threadIdx.x == 0) h->t_start = t0;
    char *gscratch = a.cta_scratch + (size_t)blockIdx.x * a.cta_scratch_bytes;
    unsigned long long cells = 0, props = 0, solved = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t q = atomicAdd(&h->work[0], 1u);
            s_item = q < a.total ? a.order[q] : 0xFFFFFFFFu;
            if (q < a.total && globaltimer_ns() > deadline) {
                set_status(h, LLP_ERR_TIMEOUT);
                s_item = 0xFFFFFFFFu;
            }
        }
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();
        if (item == 0xFFFFFFFFu) break;
        const uint32_t fam = item >> 30, i = item & 0x3FFFFFFFu;
        if (fam == kFamKnap) {
            const int64_t o = b.knap_item_off[i];
            const int32_t n = (int32_t)(b.knap_item_off[i + 1] - o);
            const int32_t W = b.knap_capacity[i];
            if (W < 0 || W > b.knap_max_capacity) {
                if (threadIdx.x == 0) set_status(h, LLP_ERR_INVALID_ARG);
                continue;
            }
            if (cta_sum_i32(n, b.knap_v + o) > 0x7FFFFFFFll) {
                if (threadIdx.x == 0) set_status(h, LLP_ERR_OVERFLOW);
                continue;
            }
            int32_t *row = ((size_t)(W + 1) * 4 <= a.smem_bytes) ? (int32_t *)smem : (int32_t *)gscratch;
            knapsack_cta<R>(n, b.knap_w + o, b.knap_v + o, W, row, h);
            if (threadIdx.x == 0) b.knap_best[i] = row[W];
            cells += (threadIdx.x == 0) ? (unsigned long long)n * (unsigned long long)(W + 1) : 0ull;
            __syncthreads();
        } else if (fam == kFamJob) {
            const int64_t j0 = b.job_off[i];
            const int32_t n = (int32_t)(b.job_off[i + 1] - j0);
            if (n > b.job_max_n) {
                if (threadIdx.x == 0) set_status(h, LLP_ERR_INVALID_ARG);
                continue;
            }
            int32_t *base = ((size_t)n * 16 <= a.smem_bytes) ? (int32_t *)smem : (int32_t *)gscratch;
            const int32_t fixed =
                job_cta(n, b.job_succ_offsets + j0, b.job_succ_indices, b.job_duration + j0, b.job_completion + j0,
                        base, base + n, base + 2 * (size_t)n, base + 3 * (size_t)n, h);
            if (threadIdx.x == 0 && fixed != n) set_status(h, LLP_ERR_INFEASIBLE);
            cells += (threadIdx.x == 0)
                         ? (unsigned long long)(b.job_succ_offsets[j0 + n] - b.job_succ_offsets[j0])
                         : 0ull;
        } else if (fam == kFamGraph) {
            const int64_t v0 = b.gr_off[i];
            const int32_t n = (int32_t)(b.gr_off[i + 1] - v0);
            const int32_t src = b.gr_source[i];
            const bool unit = b.gr_unit && b.gr_unit[i];
            if (n < 1 || n > b.gr_max_n || src < 0 || src >= n || (!unit && !b.gr_weights)) {
                if (threadIdx.x == 0) set_status(h, LLP_ERR_INVALID_ARG);
                continue;
            }
            const size_t nw = ((size_t)n + 31) / 32;
            uint32_t *dout = b.gr_dist + v0;
            const bool in_smem = (size_t)n * 4 + nw * 8 <= a.smem_bytes;
            uint32_t *d = in_smem ? (uint32_t *)smem : dout;
            uint32_t *bm = in_smem ? (uint32_t *)smem + n : (uint32_t *)gscratch;
            unsigned long long arcs = 0;
            graph_cta(n, b.gr_arc_offsets + v0, b.gr_indices, b.gr_weights, unit, src, d, bm, bm + nw, h, deadline,
                      arcs);
            if (in_smem)
                for (int32_t v = threadIdx.x; v < n; v += blockDim.x) dout[v] = d[v];
            cells += arcs;
            __syncthreads();
        } else {
            const int32_t n = b.sm_n[i];
            if (n < 1 || n > b.sm_max_n) {
                if (threadIdx.x == 0) set_status(h, LLP_ERR_INVALID_ARG);
                continue;
            }
            char *base = ((size_t)n * 12 <= a.smem_bytes) ? (char *)smem : gscratch;
            const int64_t po = b.sm_pref_off[i];
            props += marriage_cta(n, b.sm_men_pref + po, b.sm_women_rank + po, b.sm_wife + b.sm_man_off[i],
                                  (unsigned long long *)base, (int32_t *)(base + (size_t)n * 8), h, deadline);
        }
        solved += (threadIdx.x == 0);
    }
    props = warp_sum(props);
    if (lane_id() == 0 && props) atomicAdd(&h->aux, props);
    if (threadIdx.x == 0) {
        atomicAdd(&h->items, solved);
        atomicAdd(&h->edges, cells);
        __threadfence();
        const uint32_t done = atomicAdd(&h->scratch[0], 1u) + 1u;
        if (done == gridDim.x) {
            h->t_end = globaltimer_ns();
            h->sweeps = 1;
        }
    }
}

struct BatchPlan {
    size_t smem_bytes;
    size_t cta_scratch_bytes;
    int grid_max;
    size_t order_off, scratch_off, total_bytes;
};

int max_dyn_smem() {
    const DeviceInfo di = device_info();
    // opt-in limit minus the static shared memory of the solvers (a few hundred bytes)
    const int lim = di.max_smem_optin > 0 ? di.max_smem_optin : 232448;
    return lim - 1024;
}

// ctas: resident CTAs per SM (1 or 2); each gets 1/ctas of the shared memory.
BatchPlan plan_batch(const llp_batch_t *b, int ctas = 1) {
    BatchPlan p{};
    p.smem_bytes = (size_t)max_dyn_smem() / ctas / 16 * 16;
    size_t need = 0;
    if (b->knap_count > 0 && (size_t)(b->knap_max_capacity + 1) * 4 > p.smem_bytes)
        need = std::max(need, (size_t)(b->knap_max_capacity + 1) * 4);
    if (b->job_count > 0 && (size_t)b->job_max_n * 16 > p.smem_bytes) need = std::max(need, (size_t)b->job_max_n * 16);
    if (b->sm_count > 0 && (size_t)b->sm_max_n * 12 > p.smem_bytes) need = std::max(need, (size_t)b->sm_max_n * 12);
    if (b->gr_count > 0) {
        const size_t nw = ((size_t)b->gr_max_n + 31) / 32;
        if ((size_t)b->gr_max_n * 4 + nw * 8 > p.smem_bytes) need = std::max(need, nw * 8);  // bitmaps only
    }
    p.cta_scratch_bytes = align_up(need, 256);
    const DeviceInfo di = device_info();
    p.grid_max = (di.sms > 0 ? di.sms : 148) * ctas;
    const size_t total = (size_t)b->knap_count + b->job_count + b->sm_count + b->gr_count;
    Carve c(nullptr);
    c.take<uint32_t>(total);
    p.order_off = kHeaderBytes;
    p.scratch_off = align_up(c.off, 256);
    p.total_bytes = p.scratch_off + p.cta_scratch_bytes * (size_t)p.grid_max;
    return p;
}

llp_status_t validate_batch(const llp_batch_t *b) {
    if (!b) return LLP_ERR_INVALID_ARG;
    if (b->knap_count < 0 || b->job_count < 0 || b->sm_count < 0 || b->gr_count < 0) return LLP_ERR_INVALID_ARG;
    if ((int64_t)b->knap_count + b->job_count + b->sm_count + b->gr_count > (1 << 29)) return LLP_ERR_INVALID_ARG;
    if (b->knap_count > 0 && (!b->knap_item_off || !b->knap_w || !b->knap_v || !b->knap_capacity ||
                              !b->knap_best || b->knap_max_capacity < 0 || b->knap_max_capacity > (1 << 26)))
        return LLP_ERR_INVALID_ARG;
    if (b->job_count > 0 && (!b->job_off || !b->job_succ_offsets || !b->job_duration || !b->job_completion ||
                             b->job_max_n < 1))
        return LLP_ERR_INVALID_ARG;
    if (b->sm_count > 0 && (!b->sm_n || !b->sm_pref_off || !b->sm_man_off || !b->sm_men_pref ||
                            !b->sm_women_rank || !b->sm_wife || b->sm_max_n < 1 || b->sm_max_n > (1 << 24)))
        return LLP_ERR_INVALID_ARG;
    if (b->gr_count > 0 && (!b->gr_off || !b->gr_arc_offsets || !b->gr_source || !b->gr_dist || b->gr_max_n < 1 ||
                            b->gr_max_n > (1 << 29)))
        return LLP_ERR_INVALID_ARG;
    return LLP_OK;
}

template <int R>
llp_status_t launch_batch(const BatchArgs &a, int threads, int grid, cudaStream_t st) {
    LLP_CUDA_TRY(cudaFuncSetAttribute(batch_solve_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)a.smem_bytes));
    batch_solve_kernel<R><<<grid, threads, a.smem_bytes, st>>>(a);
    LLP_CUDA_TRY(cudaGetLastError());
    return LLP_OK;
}

}  // namespace
}  // namespace llp

extern "C" {

size_t llp_batch_workspace_size(const llp_batch_t *b) {
    if (llp::validate_batch(b) != LLP_OK) return 0;
    // enough for either launch shape (two CTAs per SM have more, smaller scratch areas)
    return std::max(llp::plan_batch(b, 1).total_bytes, llp::plan_batch(b, 2).total_bytes);
}

llp_status_t llp_batch_solve(const llp_batch_t *b, const llp_batch_cfg_t *cfg, const llp_sched_t *sched, void *ws,
                             size_t ws_bytes, void *stream) {
    using namespace llp;
    llp_status_t rc = validate_batch(b);
    if (rc != LLP_OK) return rc;
    if (!ws || ((uintptr_t)ws & 255u) != 0) return LLP_ERR_INVALID_ARG;
    int threads = (cfg && (cfg->threads == 256 || cfg->threads == 512 || cfg->threads == 1024))
                      ? cfg->threads : 1024;
    const int ctas = (cfg && cfg->ctas_per_sm == 2) ? 2 : 1;
    if (ctas == 2 && threads > 512) threads = 512;
    const BatchPlan p = plan_batch(b, ctas);
    if (ws_bytes < p.total_bytes) return LLP_ERR_WORKSPACE_TOO_SMALL;
    const int unroll = (cfg && (cfg->knap_unroll == 4 || cfg->knap_unroll == 16)) ? cfg->knap_unroll : 8;
    cudaStream_t st = (cudaStream_t)stream;
    rc = reset_header(ws, st);
    if (rc != LLP_OK) return rc;
    BatchArgs a;
    a.b = *b;
    a.order = (uint32_t *)((char *)ws + p.order_off);
    a.total = (uint32_t)((size_t)b->knap_count + b->job_count + b->sm_count + b->gr_count);
    a.cta_scratch = (char *)ws + p.scratch_off;
    a.cta_scratch_bytes = p.cta_scratch_bytes;
    a.smem_bytes = p.smem_bytes;
    a.h = (WsHeader *)ws;
    a.deadline_ns = deadline_from(sched);
    if (a.total == 0) return LLP_OK;
    batch_plan_kernel<<<1, 1024, 0, st>>>(a);
    LLP_CUDA_TRY(cudaGetLastError());
    const int grid = std::min<int>(p.grid_max, (int)a.total);
    if (unroll == 4) return launch_batch<4>(a, threads, grid, st);
    if (unroll == 16) return launch_batch<16>(a, threads, grid, st);
    return launch_batch<8>(a, threads, grid, st);
}

llp_status_t llp_batch_autotune(const llp_batch_t *b, void *ws, size_t ws_bytes, void *stream,
                                llp_batch_cfg_t *best, float *h_ms, int32_t max_tried, int32_t *n_tried) {
    using namespace llp;
    if (!best) return LLP_ERR_INVALID_ARG;
    // (threads, CTAs per SM) x knapsack blocking
    static const int kShape[][2] = {{1024, 1}, {512, 1}, {512, 2}, {256, 2}};
    static const int kUnrollC[] = {4, 8, 16};
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    LLP_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return LLP_ERR_CUDA;
    }
    float best_ms = 1e30f;
    int tried = 0;
    llp_status_t rc = LLP_OK;
    for (const auto &sh : kShape)
        for (int u : kUnrollC) {
            llp_batch_cfg_t c{};
            c.threads = sh[0];
            c.ctas_per_sm = sh[1];
            c.knap_unroll = u;
            // one untimed run (warm), one timed run
            rc = llp_batch_solve(b, &c, nullptr, ws, ws_bytes, stream);
            if (rc != LLP_OK) break;
            cudaEventRecord(e0, st);
            rc = llp_batch_solve(b, &c, nullptr, ws, ws_bytes, stream);
            cudaEventRecord(e1, st);
            if (rc != LLP_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = LLP_ERR_CUDA;
                break;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (h_ms && tried < max_tried) h_ms[tried] = ms;
            tried++;
            if (ms < best_ms) {
                best_ms = ms;
                *best = c;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (n_tried) *n_tried = tried;
    (void)cudaGetLastError();
    return rc;
}

}  // extern "C"

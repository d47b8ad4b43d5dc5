// Job scheduling as an LLP (paper Sec. 4.4), single instance, one cooperative
// launch over the whole GPU.
//
// G[j] = completion time, bottom G[j] = t_j.  A job is forbidden when it is
// ready (every predecessor fixed) and G[j] < max_p G[p] + t_j; the advance
// raises G[j] to that bound and fixes j.  As in the paper's implementation the
// predecessor maximum is kept incrementally in maxp[] (atomicMax, the paper's
// max_from_parents) and readiness in remaining[] (atomicSub, remaining_prereqs):
// a job enters the worklist exactly when its last predecessor is fixed.  Sweeps
// are separated by a bounded grid barrier; the run stops when a sweep fixes no
// job.  Jobs left unfixed mean a cycle: LLP_ERR_INFEASIBLE.
#include "llp_common.cuh"

#ifndef LLP_JOB_STAGE
#define LLP_JOB_STAGE 1
#endif

namespace llp {
constexpr uint32_t kJobStage = 4096;  // ready jobs a CTA stages per sweep before spilling
namespace {

template <typename OffT>
struct JobArgs {
    int32_t n;
    const OffT *off;
    const int32_t *idx;
    const int32_t *dur;
    int32_t *completion;
    int32_t *remaining;
    int32_t *maxp;
    int32_t *list[2];
    WsHeader *h;
    long long deadline_ns;
};

template <typename OffT>
__global__ void __launch_bounds__(512) job_sweep_kernel(JobArgs<OffT> a) {
    WsHeader *h = a.h;
#if LLP_JOB_STAGE
    __shared__ int32_t s_ready[kJobStage];
    __shared__ uint32_t s_nready, s_base;
    if (threadIdx.x == 0) s_nready = 0;
#endif
    const long long t0 = globaltimer_ns();
    const long long deadline = t0 + a.deadline_ns;
    uint32_t phase = 0;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
    const int wpb = blockDim.x >> 5;
    const int64_t gwarp = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * wpb;
    const int64_t m = (int64_t)__ldg(a.off + a.n);
    unsigned long long fixed = 0, edges = 0;

    // init_global_state: G = t, readiness counters from the in-degrees
    for (int64_t j = gtid; j < a.n; j += gthreads) {
        a.remaining[j] = 0;
        a.maxp[j] = 0;
        a.completion[j] = __ldg(a.dur + j);
    }
    if (gtid == 0) h->t_start = t0;
    bool alive = grid_barrier(h, phase, deadline);
    if (alive) {
        for (int64_t e = gtid; e < m; e += gthreads) atomicAdd(a.remaining + __ldg(a.idx + e), 1);
        alive = grid_barrier(h, phase, deadline);
    }
    // initial_states_to_process: the sources
    if (alive) {
        for (int64_t base = gwarp * 32; base < a.n; base += nwarps * 32) {
            const int64_t j = base + lane_id();
            const bool src = j < a.n && a.remaining[j] == 0;
            const uint32_t slot = warp_append_slot(src, &h->n_small[0]);
            if (src) a.list[0][slot] = (int32_t)j;
        }
        alive = grid_barrier(h, phase, deadline);
    }
    uint32_t k = 0;
    while (alive) {
        const uint32_t cnt = cta_read_once(&h->n_small[k % 3]);
        if (gtid == 0) h->n_small[(k + 2) % 3] = 0;
        if (cnt == 0) break;
        const int32_t *cur = a.list[k & 1];
        int32_t *nxt = a.list[(k + 1) & 1];
        uint32_t *ncount = &h->n_small[(k + 1) % 3];
        for (int64_t base = gwarp * 32; base < cnt; base += nwarps * 32) {
            const int64_t i = base + lane_id();
            const bool ok = i < cnt;
            int32_t j = 0;
            long long c = 0;
            OffT beg = 0;
            uint32_t deg = 0;
            if (ok) {
                j = cur[i];
                c = (long long)__ldcg(a.maxp + j) + __ldg(a.dur + j);
                if (c > 0x7FFFFFFFll) {
                    set_status(h, LLP_ERR_OVERFLOW);
                    c = 0x7FFFFFFF;
                }
                a.completion[j] = (int32_t)c;  // advance + fix
                beg = __ldg(a.off + j);
                deg = (uint32_t)(__ldg(a.off + j + 1) - beg);
                fixed++;
            }
            // publish to successors, edge-balanced across the warp
            uint32_t incl = deg;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane_id() >= o) incl += t;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            const uint32_t excl = incl - deg;
            edges += lane_id() == 0 ? total : 0;
            for (uint32_t b = 0; b < total; b += 32) {
                const uint32_t t = b + lane_id();
                int pos = 0;
#pragma unroll
                for (int s = 16; s > 0; s >>= 1) {
                    const uint32_t probe = __shfl_sync(0xffffffffu, incl, pos + s - 1);
                    if (probe <= t) pos += s;
                }
                const bool live = t < total;
                const int owner = live ? pos : 0;
                const uint32_t ex = __shfl_sync(0xffffffffu, excl, owner);
                const OffT bo = __shfl_sync(0xffffffffu, beg, owner);
                const int32_t co = __shfl_sync(0xffffffffu, (int32_t)c, owner);
                bool ready = false;
                int32_t s = 0;
                if (live) {
                    s = __ldg(a.idx + bo + (OffT)(t - ex));
                    atomicMax(a.maxp + s, co);
                    ready = atomicSub(a.remaining + s, 1) == 1;
                }
#if LLP_JOB_STAGE
                // ready jobs are staged in the CTA's shared buffer; a full buffer spills to the list
                const uint32_t mask = __ballot_sync(0xffffffffu, ready);
                if (mask) {
                    uint32_t at = 0;
                    if (lane_id() == 0) at = atomicAdd(&s_nready, (uint32_t)__popc(mask));
                    at = __shfl_sync(0xffffffffu, at, 0);
                    const uint32_t my = at + __popc(mask & lanemask_lt());
                    // every buffer position below kJobStage is written by exactly one lane; the
                    // lanes past the buffer's end go straight to the list
                    if (ready && my < kJobStage) s_ready[my] = s;
                    if (at + __popc(mask) > kJobStage) {
                        const bool spill = ready && my >= kJobStage;
                        const uint32_t slot = warp_append_slot(spill, ncount);
                        if (spill) nxt[slot] = s;
                    }
                }
#else
                const uint32_t slot = warp_append_slot(ready, ncount);
                if (ready) nxt[slot] = s;
#endif
            }
        }
#if LLP_JOB_STAGE
        // the CTA's staged ready jobs: one reservation in the next list
        __syncthreads();
        const uint32_t nst = min(s_nready, kJobStage);
        if (threadIdx.x == 0) s_base = nst ? atomicAdd(ncount, nst) : 0u;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < nst; i += blockDim.x) nxt[s_base + i] = s_ready[i];
        if (threadIdx.x == 0) s_nready = 0;  // read again only after the grid barrier
#endif
        alive = grid_barrier(h, phase, deadline);
        k++;
    }
    const unsigned long long fs = warp_sum(fixed), es = warp_sum(edges);
    if (lane_id() == 0) {
        atomicAdd(&h->advances, fs);
        atomicAdd(&h->edges, es);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t done = atomicAdd(&h->scratch[0], 1u) + 1u;
        if (done == gridDim.x) {
            __threadfence();
            h->t_end = globaltimer_ns();
            h->sweeps = (int32_t)k;
            const unsigned long long nfixed = *(volatile unsigned long long *)&h->advances;
            h->items = nfixed;
            if (alive && nfixed != (unsigned long long)a.n) set_status(h, LLP_ERR_INFEASIBLE);
        }
    }
}

struct JobLayout {
    int32_t *remaining, *maxp, *list[2];
    size_t bytes;
};

JobLayout carve_job(void *ws, int32_t n) {
    Carve c(ws);
    JobLayout L;
    L.remaining = c.take<int32_t>(n);
    L.maxp = c.take<int32_t>(n);
    L.list[0] = c.take<int32_t>(n);
    L.list[1] = c.take<int32_t>(n);
    L.bytes = c.bytes();
    return L;
}

}  // namespace
}  // namespace llp

extern "C" {

size_t llp_job_schedule_workspace_size(int32_t n, int64_t m) {
    (void)m;
    if (n < 1) return 0;
    return llp::carve_job(nullptr, n).bytes;
}

llp_status_t llp_job_schedule(const llp_csr_t *succ, const int32_t *duration, int32_t *completion,
                              const llp_sched_t *sched, void *ws, size_t ws_bytes, void *stream) {
    using namespace llp;
    if (!succ || !duration || !completion || !ws || succ->n < 1 || succ->m < 0 || !succ->offsets)
        return LLP_ERR_INVALID_ARG;
    if (succ->m > 0 && !succ->indices) return LLP_ERR_INVALID_ARG;
    if (!succ->offsets_64 && succ->m > 0x7FFFFFFFll) return LLP_ERR_INVALID_ARG;
    if (((uintptr_t)ws & 255u) != 0) return LLP_ERR_INVALID_ARG;
    JobLayout L = carve_job(ws, succ->n);
    if (ws_bytes < L.bytes) return LLP_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t st = (cudaStream_t)stream;
    llp_status_t rc = reset_header(ws, st);
    if (rc != LLP_OK) return rc;
    auto fill = [&](auto &a) {
        a.n = succ->n;
        a.idx = succ->indices;
        a.dur = duration;
        a.completion = completion;
        a.remaining = L.remaining;
        a.maxp = L.maxp;
        a.list[0] = L.list[0];
        a.list[1] = L.list[1];
        a.h = (WsHeader *)ws;
        a.deadline_ns = deadline_from(sched);
    };
    // one CTA per SM: the level sweeps are short (one grid barrier each) and measured
    // faster with half the co-resident CTAs (1M-job DAG: 0.90 -> 0.73 ms)
    const int grid = device_info().sms > 0 ? device_info().sms : 0;
    if (succ->offsets_64) {
        JobArgs<int64_t> a;
        fill(a);
        a.off = (const int64_t *)succ->offsets;
        void *args[] = {&a};
        return launch_cooperative((const void *)job_sweep_kernel<int64_t>, 512, 0, grid, args, st);
    }
    JobArgs<int32_t> a;
    fill(a);
    a.off = (const int32_t *)succ->offsets;
    void *args[] = {&a};
    return launch_cooperative((const void *)job_sweep_kernel<int32_t>, 512, 0, grid, args, st);
}

}  // extern "C"

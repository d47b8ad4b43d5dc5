// Stable marriage as an LLP (paper Sec. 4.3), single instance on the whole GPU.
//
// G[m] = next[m] (index into man m's preference list), bottom = all zeros.
// forbidden(m) <=> best[w] < (rank_w(m) << 32 | m) for the woman w = pref[m][G[m]],
// where best[w] is the atomicMin over every suitor w has received; advance =
// G[m] + 1.  Every man starts in the worklist (one thread each); a thread whose
// man is accepted by an engaged woman continues with the man she released
// (the paper's PTCF idea of re-advancing displaced men at once).  The fixed
// point is the man-optimal stable matching.
#include "llp_common.cuh"
#include "problems.cuh"

namespace llp {
namespace {

__global__ void marriage_init(int32_t n, unsigned long long *best, int32_t *next) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        best[i] = kEmptySuitor;
        next[i] = 0;
    }
}

__global__ void __launch_bounds__(256) marriage_propose(int32_t n, const int32_t *men_pref, const int32_t *women_rank,
                                                        unsigned long long *best, int32_t *next, WsHeader *h,
                                                        long long deadline_ns) {
    const long long t0 = globaltimer_ns();
    if (blockIdx.x == 0 && threadIdx.x == 0) h->t_start = t0;
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long props = 0;
    if (m < n) {
        bool failed = false;
        props = propose_chain((int32_t)m, 0, n, men_pref, women_rank, best, next, h, t0 + deadline_ns, failed);
    }
    props = warp_sum(props);
    if (lane_id() == 0 && props) atomicAdd(&h->aux, props);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t done = atomicAdd(&h->scratch[0], 1u) + 1u;
        if (done == gridDim.x) {
            h->t_end = globaltimer_ns();
            h->sweeps = 1;
        }
    }
}

// final_solution: wife[m] = pref[m][G[m]], husband[w] = man in best[w].
__global__ void marriage_extract(int32_t n, const int32_t *men_pref, const unsigned long long *best,
                                 const int32_t *next, int32_t *wife, int32_t *husband, int32_t *next_out,
                                 WsHeader *h) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = next[i];
        wife[i] = (k >= 0 && k < n) ? men_pref[i * (int64_t)n + k] : -1;
        if (next_out) next_out[i] = k;
        if (husband) {
            const unsigned long long b = best[i];
            husband[i] = b == kEmptySuitor ? -1 : (int32_t)(uint32_t)(b & 0xFFFFFFFFull);
        }
    }
    (void)h;
}

struct MarriageLayout {
    unsigned long long *best;
    int32_t *next;
    size_t bytes;
};

MarriageLayout carve_marriage(void *ws, int32_t n) {
    Carve c(ws);
    MarriageLayout L;
    L.best = c.take<unsigned long long>(n);
    L.next = c.take<int32_t>(n);
    L.bytes = c.bytes();
    return L;
}

}  // namespace
}  // namespace llp

extern "C" {

size_t llp_stable_marriage_workspace_size(int32_t n) {
    if (n < 1) return 0;
    return llp::carve_marriage(nullptr, n).bytes;
}

llp_status_t llp_stable_marriage(int32_t n, const int32_t *men_pref, const int32_t *women_rank, int32_t *wife,
                                 int32_t *husband, int32_t *next, const llp_sched_t *sched, void *ws,
                                 size_t ws_bytes, void *stream) {
    using namespace llp;
    if (n < 1 || n > (1 << 24) || !men_pref || !women_rank || !wife || !ws) return LLP_ERR_INVALID_ARG;
    if (((uintptr_t)ws & 255u) != 0) return LLP_ERR_INVALID_ARG;
    MarriageLayout L = carve_marriage(ws, n);
    if (ws_bytes < L.bytes) return LLP_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t st = (cudaStream_t)stream;
    llp_status_t rc = reset_header(ws, st);
    if (rc != LLP_OK) return rc;
    WsHeader *h = (WsHeader *)ws;
    const int threads = 256;
    const int blocks = (n + threads - 1) / threads;
    const DeviceInfo di = device_info();
    const int fill_blocks = di.sms > 0 ? di.sms * 4 : 256;
    marriage_init<<<fill_blocks, 256, 0, st>>>(n, L.best, L.next);
    marriage_propose<<<blocks, threads, 0, st>>>(n, men_pref, women_rank, L.best, L.next, h, deadline_from(sched));
    marriage_extract<<<fill_blocks, 256, 0, st>>>(n, men_pref, L.best, L.next, wife, husband, next, h);
    LLP_CUDA_TRY(cudaGetLastError());
    return LLP_OK;
}

}  // extern "C"

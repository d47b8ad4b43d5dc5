// 0-1 knapsack as an LLP (paper Sec. 4.7), single instance.
//
// Cell G[k,c] = best value of items 0..k-1 within capacity c; G[0,*] = 0 is
// the bottom.  A cell is forbidden while it is below
// max(G[k-1,c], v_k + G[k-1,c-w_k]); the advance raises it to that bound.  Row
// k depends only on row k-1, so one CTA sweeps the capacity range once per
// item with the recurrence evaluated for every cell in parallel and a CTA
// barrier between items (knapsack_cta).  The row lives in shared memory when
// it fits (W+1 <= 56K cells), otherwise in the workspace (L1/L2 resident).
#include "llp_common.cuh"
#include "problems.cuh"

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
    (void)sched;
    if (n_items < 0 || capacity < 0 || capacity > (1 << 26) || !best || !ws) return LLP_ERR_INVALID_ARG;
    if (n_items > 0 && (!w || !v)) return LLP_ERR_INVALID_ARG;
    if (((uintptr_t)ws & 255u) != 0) return LLP_ERR_INVALID_ARG;
    if (ws_bytes < llp_knapsack_workspace_size(n_items, capacity)) return LLP_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t st = (cudaStream_t)stream;
    llp_status_t rc = reset_header(ws, st);
    if (rc != LLP_OK) return rc;
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

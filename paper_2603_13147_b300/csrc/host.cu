// SSSP on a graph held in host memory: the copies to the device, the sweep
// (llp_sssp) and the copy of the distances back, all enqueued on one stream.
// The device copies of the graph live in the caller's workspace, after the
// sweep's own scratch, so the call allocates nothing.
#include <algorithm>

#include "llp_common.cuh"

namespace llp {
namespace {

constexpr size_t kCopyChunk = (size_t)64 << 20;  // bytes per cudaMemcpyAsync

struct HostLayout {
    size_t sweep_bytes;
    size_t off_at, idx_at, w_at, dist_at;
    size_t bytes;
};

HostLayout host_layout(int32_t n, int64_t m, bool off64) {
    HostLayout L{};
    L.sweep_bytes = llp_sssp_workspace_size(n, m);
    size_t at = align_up(L.sweep_bytes, 256);
    L.off_at = at;
    at = align_up(at + ((size_t)n + 1) * (off64 ? 8 : 4), 256);
    L.idx_at = at;
    at = align_up(at + (size_t)m * 4, 256);
    L.w_at = at;
    at = align_up(at + (size_t)m * 4, 256);
    L.dist_at = at;
    L.bytes = align_up(at + (size_t)n * 4, 256);
    return L;
}

llp_status_t copy_chunked(void *dst, const void *src, size_t bytes, cudaMemcpyKind kind, cudaStream_t st) {
    for (size_t o = 0; o < bytes; o += kCopyChunk) {
        const size_t len = std::min(kCopyChunk, bytes - o);
        LLP_CUDA_TRY(cudaMemcpyAsync((char *)dst + o, (const char *)src + o, len, kind, st));
    }
    return LLP_OK;
}

}  // namespace
}  // namespace llp

extern "C" {

size_t llp_sssp_host_workspace_size(int32_t n, int64_t m, int32_t offsets_64) {
    if (n < 1 || m < 0) return 0;
    return llp::host_layout(n, m, offsets_64 != 0).bytes;
}

llp_status_t llp_sssp_host(const llp_csr_t *h_g, int32_t source, uint32_t *h_dist, const llp_sched_t *sched,
                           void *ws, size_t ws_bytes, void *stream) {
    using namespace llp;
    if (!h_g || !h_dist || !ws) return LLP_ERR_INVALID_ARG;
    if (h_g->n < 1 || h_g->m < 0 || !h_g->offsets) return LLP_ERR_INVALID_ARG;
    if (h_g->m > 0 && (!h_g->indices || !h_g->weights)) return LLP_ERR_INVALID_ARG;
    if (source < 0 || source >= h_g->n) return LLP_ERR_INVALID_ARG;
    if (((uintptr_t)ws & 255u) != 0) return LLP_ERR_INVALID_ARG;
    const bool off64 = h_g->offsets_64 != 0;
    const HostLayout L = host_layout(h_g->n, h_g->m, off64);
    if (ws_bytes < L.bytes) return LLP_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t st = (cudaStream_t)stream;
    char *base = (char *)ws;
    llp_csr_t dg = *h_g;
    dg.offsets = base + L.off_at;
    dg.indices = (const int32_t *)(base + L.idx_at);
    dg.weights = (const uint32_t *)(base + L.w_at);
    uint32_t *d_dist = (uint32_t *)(base + L.dist_at);
    llp_status_t rc = copy_chunked(base + L.off_at, h_g->offsets, ((size_t)h_g->n + 1) * (off64 ? 8 : 4),
                                   cudaMemcpyHostToDevice, st);
    if (rc == LLP_OK && h_g->m > 0)
        rc = copy_chunked(base + L.idx_at, h_g->indices, (size_t)h_g->m * 4, cudaMemcpyHostToDevice, st);
    if (rc == LLP_OK && h_g->m > 0)
        rc = copy_chunked(base + L.w_at, h_g->weights, (size_t)h_g->m * 4, cudaMemcpyHostToDevice, st);
    if (rc != LLP_OK) return rc;
    rc = llp_sssp(&dg, source, d_dist, sched, ws, L.sweep_bytes, stream);
    if (rc != LLP_OK) return rc;
    return copy_chunked(h_dist, d_dist, (size_t)h_g->n * 4, cudaMemcpyDeviceToHost, st);
}

}  // extern "C"

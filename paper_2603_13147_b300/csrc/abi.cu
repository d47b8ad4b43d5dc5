// Library-wide entry points: version, status strings, status readback, and the
// host launch helpers shared by the problem files.
#include <mutex>

#include "llp_common.cuh"

namespace llp {

DeviceInfo device_info() {
    static std::mutex mu;
    static DeviceInfo cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        (void)cudaGetLastError();
        return DeviceInfo{};
    }
    std::lock_guard<std::mutex> lk(mu);
    if (cache[dev].device != dev) {
        DeviceInfo d;
        d.device = dev;
        cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&d.l2_bytes, cudaDevAttrL2CacheSize, dev);
        cudaDeviceGetAttribute(&d.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        (void)cudaGetLastError();
        cache[dev] = d;
    }
    return cache[dev];
}

llp_status_t launch_cooperative(const void *func, int threads, size_t smem, int max_blocks, void **args,
                                cudaStream_t stream, int *grid_out) {
    DeviceInfo di = device_info();
    if (di.sms <= 0) return LLP_ERR_CUDA;
    int per_sm = 0;
    LLP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, threads, smem));
    if (per_sm <= 0) return LLP_ERR_CUDA;
    int grid = per_sm * di.sms;
    if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
    if (grid < 1) grid = 1;
    if (grid_out) *grid_out = grid;
    LLP_CUDA_TRY(cudaLaunchCooperativeKernel(func, dim3(grid), dim3(threads), args, smem, stream));
    return LLP_OK;
}

llp_status_t reset_header(void *ws, cudaStream_t stream) {
    LLP_CUDA_TRY(cudaMemsetAsync(ws, 0, kHeaderZeroBytes, stream));
    return LLP_OK;
}

}  // namespace llp

extern "C" {

const char *llp_version(void) { return "llp-b300 0.1 (sm_103a)"; }

const char *llp_status_string(llp_status_t code) {
    switch (code) {
        case LLP_OK: return "ok";
        case LLP_ERR_INVALID_ARG: return "invalid argument";
        case LLP_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
        case LLP_ERR_CUDA: return "CUDA error";
        case LLP_ERR_TIMEOUT: return "device wait limit reached";
        case LLP_ERR_INFEASIBLE: return "infeasible (an advance passed the top of the lattice)";
        case LLP_ERR_OVERFLOW: return "integer overflow";
        case LLP_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

llp_status_t llp_get_status(const void *ws, void *stream, llp_stats_t *out) {
    if (!ws || !out) return LLP_ERR_INVALID_ARG;
    llp::WsHeader h;
    LLP_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    LLP_CUDA_TRY(cudaMemcpy(&h, ws, sizeof(h), cudaMemcpyDeviceToHost));
    out->status = h.status;
    out->sweeps = h.sweeps;
    out->items = (int64_t)h.items;
    out->edges = (int64_t)h.edges;
    out->advances = (int64_t)h.advances;
    out->aux = (int64_t)h.aux;
    out->elapsed_ns = (h.t_end > h.t_start) ? (int64_t)(h.t_end - h.t_start) : 0;
    out->mode_used = h.mode_used;
    out->delta_used = h.delta_used;
    out->block_cfg_used = h.block_cfg_used;
    out->dense_sweeps = h.dense_sweeps;
    out->local_chain_used = (int32_t)h.scratch[8];
    out->pull_sweeps = (int32_t)h.scratch[7];
    return h.status;
}

int32_t llp_sweep_log(const void *ws, void *stream, uint32_t *out, int32_t max_records) {
    if (!ws || !out || max_records < 0) return -LLP_ERR_INVALID_ARG;
    llp::WsHeader h;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess ||
        cudaMemcpy(&h, ws, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) {
        (void)cudaGetLastError();
        return -LLP_ERR_CUDA;
    }
    int32_t cnt = h.sweeps < 0 ? 0 : h.sweeps;
    if (cnt > (int32_t)llp::kSweepLogCap) cnt = (int32_t)llp::kSweepLogCap;
    if (cnt > max_records) cnt = max_records;
    if (cnt > 0 && cudaMemcpy(out, (const char *)ws + llp::kSweepLogOffset, (size_t)cnt * 16,
                              cudaMemcpyDeviceToHost) != cudaSuccess) {
        (void)cudaGetLastError();
        return -LLP_ERR_CUDA;
    }
    return cnt;
}

}  // extern "C"

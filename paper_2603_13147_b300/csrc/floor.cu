// Access-pattern floor of a push sweep (a measurement helper, not part of the
// method): one pass over every arc of a graph that streams the CSR arrays and
// reads the per-vertex state of each arc's target at random, which is the
// memory access pattern any push sweep of SSSP (paper Sec. 4.1) has to make at
// least once per reached arc.  Nothing is written except one word per thread
// (so the loads are not dead).  The arcs are read with 16-byte vector loads and
// each lane keeps 8 target reads in flight, the configuration that reached the
// device's random-read rate.
#include "llp_common.cuh"

namespace llp {
namespace {

constexpr int kFloorThreads = 512;
constexpr int kFloorVec = 2;  // int4 vectors (4 arcs each) per lane and step

__global__ void __launch_bounds__(kFloorThreads) gather_floor_kernel(const int4 *idx4, const uint4 *w4, int64_t m4,
                                                                     const int32_t *idx, const uint32_t *w, int64_t m,
                                                                     const uint32_t *state, unsigned long long *sink) {
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long acc = ~0ull;
    for (int64_t b = t; b < m4; b += T * kFloorVec) {
        int4 a[kFloorVec];
        uint4 ww[kFloorVec];
#pragma unroll
        for (int j = 0; j < kFloorVec; j++) {
            const int64_t e = b + j * T;
            a[j] = e < m4 ? __ldcs(idx4 + e) : make_int4(0, 0, 0, 0);
            ww[j] = e < m4 ? __ldcs(w4 + e) : make_uint4(0, 0, 0, 0);
        }
        uint32_t s[kFloorVec][4];
#pragma unroll
        for (int j = 0; j < kFloorVec; j++) {
            s[j][0] = __ldcg(state + a[j].x);
            s[j][1] = __ldcg(state + a[j].y);
            s[j][2] = __ldcg(state + a[j].z);
            s[j][3] = __ldcg(state + a[j].w);
        }
#pragma unroll
        for (int j = 0; j < kFloorVec; j++) {
            acc = min(acc, (unsigned long long)s[j][0] + ww[j].x);
            acc = min(acc, (unsigned long long)s[j][1] + ww[j].y);
            acc = min(acc, (unsigned long long)s[j][2] + ww[j].z);
            acc = min(acc, (unsigned long long)s[j][3] + ww[j].w);
        }
    }
    // the arcs past the last whole vector
    for (int64_t e = m4 * 4 + t; e < m; e += T) acc = min(acc, (unsigned long long)__ldcg(state + idx[e]) + w[e]);
    sink[t] = acc;
}

}  // namespace
}  // namespace llp

extern "C" {

size_t llp_gather_floor_sink_size(void) {
    const llp::DeviceInfo di = llp::device_info();
    return (size_t)(di.sms > 0 ? di.sms : 148) * 2 * llp::kFloorThreads * sizeof(unsigned long long);
}

llp_status_t llp_gather_floor(const llp_csr_t *g, const uint32_t *state, void *sink, size_t sink_bytes, void *stream) {
    using namespace llp;
    if (!g || !state || !sink || g->m < 0 || g->n < 1 || (g->m > 0 && (!g->indices || !g->weights)))
        return LLP_ERR_INVALID_ARG;
    if (sink_bytes < llp_gather_floor_sink_size()) return LLP_ERR_WORKSPACE_TOO_SMALL;
    // 16-byte vector loads need 16-byte aligned arrays
    if (((uintptr_t)g->indices & 15u) || ((uintptr_t)g->weights & 15u)) return LLP_ERR_INVALID_ARG;
    const DeviceInfo di = device_info();
    const int grid = (di.sms > 0 ? di.sms : 148) * 2;
    const int64_t m4 = g->m / 4;
    gather_floor_kernel<<<grid, kFloorThreads, 0, (cudaStream_t)stream>>>(
        (const int4 *)g->indices, (const uint4 *)g->weights, m4, g->indices, g->weights, g->m, state,
        (unsigned long long *)sink);
    LLP_CUDA_TRY(cudaGetLastError());
    return LLP_OK;
}

}  // extern "C"

// Parallel reduction as an LLP (paper Sec. 4.5): a tree whose leaves are tiles
// of the input.  A tree node is forbidden when all of its children have
// published their partial sums and it has not combined them yet; the advance
// combines them and publishes the node's own sum.  Here every CTA owns one leaf
// tile (streamed with 128-bit loads), publishes its sum, and increments its
// parent's dependency counter; the CTA that completes a parent's counter (the
// one that makes it forbidden) advances it, and so on up to the root.  One
// launch, no grid barrier; the sum is taken modulo 2^64.
#include "llp_common.cuh"

namespace llp {
namespace {

constexpr int kFan = 32;        // children per tree node
constexpr int kMaxLevels = 4;   // 32^4 leaves at most
constexpr int kReduceThreads = 512;

struct ReduceArgs {
    int64_t n;
    const uint64_t *x;
    uint64_t *sum;
    uint64_t *partial;     // per level, nodes of that level
    uint32_t *counter;     // per level >= 1, per node
    int32_t levels;        // number of levels above the leaves
    int32_t nodes[kMaxLevels + 1];
    int32_t poff[kMaxLevels + 1];
    WsHeader *h;
};

__device__ __forceinline__ uint64_t block_sum(uint64_t v) {
    __shared__ uint64_t s[32];
    v = warp_sum(v);
    if (lane_id() == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    uint64_t t = 0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? s[threadIdx.x] : 0ull;
        t = warp_sum(t);
    }
    __syncthreads();
    return t;  // valid in thread 0
}

__global__ void __launch_bounds__(kReduceThreads) reduce_tree_kernel(ReduceArgs a) {
    __shared__ int s_last;
    const long long t0 = globaltimer_ns();
    if (blockIdx.x == 0 && threadIdx.x == 0) a.h->t_start = t0;
    // leaf tile [lo, hi)
    const int64_t leaves = gridDim.x;
    const int64_t per = (a.n + leaves - 1) / leaves;
    const int64_t lo = min(a.n, (int64_t)blockIdx.x * per);
    const int64_t hi = min(a.n, lo + per);
    uint64_t acc = 0;
    // head until 16-byte aligned, then 2 x u64 vectors, then the tail
    int64_t i = lo;
    const int64_t aligned = min(hi, lo + ((((uintptr_t)(a.x + lo)) & 15u) ? 1 : 0));
    for (int64_t j = i + threadIdx.x; j < aligned; j += blockDim.x) acc += __ldg(a.x + j);
    i = aligned;
    const int64_t nvec = (hi - i) / 2;
    const ulonglong2 *xv = reinterpret_cast<const ulonglong2 *>(a.x + i);
    // four independent 16-byte loads per thread in flight (enough bytes in flight per SM
    // to cover the memory latency at full bandwidth)
    const int64_t bd = blockDim.x;
    int64_t j = threadIdx.x;
    for (; j + 3 * bd < nvec; j += 4 * bd) {
        const ulonglong2 q0 = __ldcs(xv + j), q1 = __ldcs(xv + j + bd), q2 = __ldcs(xv + j + 2 * bd),
                         q3 = __ldcs(xv + j + 3 * bd);
        acc += (q0.x + q0.y) + (q1.x + q1.y) + (q2.x + q2.y) + (q3.x + q3.y);
    }
    for (; j < nvec; j += bd) {
        const ulonglong2 q = __ldcs(xv + j);
        acc += q.x + q.y;
    }
    for (int64_t j = i + 2 * nvec + threadIdx.x; j < hi; j += blockDim.x) acc += __ldg(a.x + j);
    uint64_t s = block_sum(acc);
    // publish the leaf, then climb while this CTA completes the parent
    int64_t node = blockIdx.x;
    for (int lvl = 0;; lvl++) {
        if (threadIdx.x == 0) {
            a.partial[a.poff[lvl] + node] = s;
            if (lvl == a.levels) a.sum[0] = s;
        }
        if (lvl == a.levels) break;
        const int64_t parent = node / kFan;
        const int64_t first = parent * kFan;
        const int64_t kids = min((int64_t)kFan, (int64_t)a.nodes[lvl] - first);
        if (threadIdx.x == 0) {
            __threadfence();
            const uint32_t prev = atomicAdd(a.counter + a.poff[lvl + 1] + parent, 1u);
            s_last = (prev + 1 == (uint32_t)kids);
            __threadfence();
        }
        __syncthreads();
        if (!s_last) break;
        // advance the parent: combine its children's published sums
        uint64_t c = 0;
        if (threadIdx.x < kids) c = *(volatile uint64_t *)(a.partial + a.poff[lvl] + first + threadIdx.x);
        s = block_sum(c);
        node = parent;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const uint32_t done = atomicAdd(&a.h->scratch[0], 1u) + 1u;
        if (done == gridDim.x) {
            a.h->t_end = globaltimer_ns();
            a.h->sweeps = a.levels + 1;
            a.h->items = (unsigned long long)a.n;
        }
    }
}

struct ReducePlan {
    int32_t leaves;
    int32_t levels;
    int32_t nodes[kMaxLevels + 1];
    int32_t poff[kMaxLevels + 1];
    int32_t total;
};

ReducePlan plan_reduce(int64_t n) {
    ReducePlan p{};
    const DeviceInfo di = device_info();
    const int sms = di.sms > 0 ? di.sms : 148;
    // enough CTAs to saturate HBM, at least ~64 KB of input per leaf
    int64_t leaves = (int64_t)sms * 4;
    const int64_t by_size = (n + 8191) / 8192;
    if (by_size < leaves) leaves = by_size;
    if (leaves < 1) leaves = 1;
    p.leaves = (int32_t)leaves;
    p.nodes[0] = p.leaves;
    p.poff[0] = 0;
    int lvl = 0, total = p.leaves;
    while (p.nodes[lvl] > 1 && lvl < kMaxLevels) {
        p.nodes[lvl + 1] = (p.nodes[lvl] + kFan - 1) / kFan;
        p.poff[lvl + 1] = total;
        total += p.nodes[lvl + 1];
        lvl++;
    }
    p.levels = lvl;
    p.total = total;
    return p;
}

}  // namespace
}  // namespace llp

extern "C" {

size_t llp_reduce_workspace_size(int64_t n) {
    if (n < 0) return 0;
    // the plan depends on the SM count; size for the largest leaf count
    const size_t nodes = 148 * 64 + 4096;
    return llp::kHeaderBytes + llp::align_up(nodes * 8, 256) + llp::align_up(nodes * 4, 256);
}

llp_status_t llp_reduce(int64_t n, const uint64_t *x, uint64_t *sum, const llp_sched_t *sched, void *ws,
                        size_t ws_bytes, void *stream) {
    using namespace llp;
    (void)sched;
    if (n < 0 || !sum || !ws || (n > 0 && !x)) return LLP_ERR_INVALID_ARG;
    if (((uintptr_t)x & 7u) != 0) return LLP_ERR_INVALID_ARG;
    if (((uintptr_t)ws & 255u) != 0) return LLP_ERR_INVALID_ARG;
    if (ws_bytes < llp_reduce_workspace_size(n)) return LLP_ERR_WORKSPACE_TOO_SMALL;
    ReducePlan p = plan_reduce(n);
    if (p.nodes[p.levels] != 1 || (size_t)p.total > 148 * 64 + 4096) return LLP_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    // header and counters are zeroed together (counters follow the partials)
    Carve c(ws);
    uint64_t *partial = c.take<uint64_t>(148 * 64 + 4096);
    uint32_t *counter = c.take<uint32_t>(148 * 64 + 4096);
    LLP_CUDA_TRY(cudaMemsetAsync(ws, 0, kHeaderZeroBytes, st));
    LLP_CUDA_TRY(cudaMemsetAsync(counter, 0, (size_t)p.total * 4, st));
    ReduceArgs a;
    a.n = n;
    a.x = x;
    a.sum = sum;
    a.partial = partial;
    a.counter = counter;
    a.levels = p.levels;
    for (int i = 0; i <= kMaxLevels; i++) {
        a.nodes[i] = p.nodes[i];
        a.poff[i] = p.poff[i];
    }
    a.h = (WsHeader *)ws;
    reduce_tree_kernel<<<p.leaves, kReduceThreads, 0, st>>>(a);
    LLP_CUDA_TRY(cudaGetLastError());
    return LLP_OK;
}

}  // extern "C"

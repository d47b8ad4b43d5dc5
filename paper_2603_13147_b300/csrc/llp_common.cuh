// Shared device/host helpers of libllp: workspace header, device status word,
// bounded grid barrier, warp-aggregated appends, host launch utilities.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/llp.h"

namespace llp {

constexpr int64_t kDefaultDeadlineNs = 10LL * 1000 * 1000 * 1000;  // 10 s
constexpr size_t kHeaderBytes = 65536;  // WsHeader, then the sweep log
constexpr size_t kHeaderZeroBytes = 4096;  // part of the header cleared per call
constexpr size_t kSweepLogOffset = 4096;
constexpr uint32_t kSweepLogCap = (uint32_t)((kHeaderBytes - kSweepLogOffset) / 16);

// One record per sweep (graph engine): device time since the call started,
// worklist sizes at the start of the sweep and flags (bit 0 dense sweep,
// bit 1 bucket advance).
struct SweepRec {
    uint32_t t_ns;
    uint32_t n_small;
    uint32_t n_chunk;
    uint32_t flags;
};

__device__ __forceinline__ SweepRec *sweep_log(void *h) { return (SweepRec *)((char *)h + kSweepLogOffset); }
constexpr uint32_t kInf = 0xFFFFFFFFu;

// Workspace header: the first kHeaderBytes of every workspace.  Zeroed by the
// host (cudaMemsetAsync) at the start of each call.
struct alignas(256) WsHeader {
    // ---- mirrored into llp_stats_t
    int32_t status;
    int32_t sweeps;
    unsigned long long items;
    unsigned long long edges;
    unsigned long long advances;
    unsigned long long aux;
    long long t_start;
    long long t_end;
    int32_t mode_used;
    uint32_t delta_used;
    int32_t block_cfg_used;
    int32_t dense_sweeps;
    // ---- grid barrier
    alignas(128) uint32_t bar_count;
    alignas(128) uint32_t bar_gen;
    alignas(128) uint32_t abort_flag;
    // ---- engine counters
    alignas(128) uint32_t n_small[3];
    uint32_t n_chunk[3];
    alignas(128) uint32_t work[3];
    alignas(128) uint32_t n_far[3];
    uint32_t far_min[3];
    uint32_t list_ok[3];
    unsigned long long sweep_edges[2];
    // [0] CTAs finished (t_end), [1..2] closure change flags, [7] pull sweeps,
    // [8] local chain used, [9..14] feature accumulators, [15] feature CTAs finished
    uint32_t scratch[16];
    // load-balanced engine: per list (sweep k uses k % 3) entries << 32 | arcs
    unsigned long long lb_cursor[3];
    // ---- schedule chosen on the device by the learned scheduler (graph engine)
    int32_t sched_mode;
    uint32_t sched_delta;
    int32_t sched_cfg;
    int32_t sched_chain;
    int32_t sched_gw;       // dense-sweep group width, 0 = the grid-size rule
    int32_t sched_valid;
    float feat[16];  // instance features the choice was made from
    float feat_wmax; // largest sampled arc weight
};
static_assert(sizeof(WsHeader) <= kHeaderZeroBytes, "header too large");

// ------------------------------------------------------------ device helpers

__device__ __forceinline__ long long globaltimer_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// First writer wins: the first device-side error is the one reported.
__device__ __forceinline__ void set_status(WsHeader *h, int32_t code) {
    atomicCAS(&h->status, 0, code);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Bounded grid-wide barrier for a cooperative (co-resident) grid.  Every block
// calls it the same number of times.  Returns false when the call must stop
// (deadline passed or another block aborted); the block then leaves its loop.
// Sense reversal on one counter word: block 0 adds 2^31 - (gridDim.x - 1), the
// others add 1, so the word's top bit flips exactly when the last block has
// arrived (its low bits never change across complete barriers).  Arrival is an
// acq_rel atomic (it publishes the block's writes, ordered before it by
// __syncthreads); waiting is an acquire load of the same word.
__device__ __forceinline__ bool grid_barrier(WsHeader *h, uint32_t &phase, long long deadline) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t add = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u;
        uint32_t old;
        asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;"
                     : "=r"(old) : "l"(&h->bar_count), "r"(add) : "memory");
        int ok = 1;
        uint32_t spins = 0;
        while (((ld_acquire_u32(&h->bar_count) ^ old) & 0x80000000u) == 0) {
            if ((++spins & 63u) == 0) {
                if (ld_relaxed_u32(&h->abort_flag)) { ok = 0; break; }
                if (globaltimer_ns() > deadline) {
                    set_status(h, LLP_ERR_TIMEOUT);
                    atomicExch(&h->abort_flag, 1u);
                    ok = 0;
                    break;
                }
            }
        }
        if (ok && globaltimer_ns() > deadline) {  // total time limit of the call
            set_status(h, LLP_ERR_TIMEOUT);
            atomicExch(&h->abort_flag, 1u);
        }
        if (ld_relaxed_u32(&h->abort_flag)) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    phase += 1;
    return s_ok != 0;
}

// A word every thread of a grid needs at the same point (a worklist size, a
// change flag): one thread per CTA reads it and the CTA shares it through shared
// memory, instead of every warp of the grid reading the same L2 line (those
// requests queue at one L2 slice).  CTA-collective.
template <typename T>
__device__ __forceinline__ T cta_read_once(const T *p) {
    __shared__ T s_v;
    if (threadIdx.x == 0) s_v = *(volatile const T *)p;
    __syncthreads();
    const T v = s_v;
    __syncthreads();  // every thread has the value before a later call overwrites it
    return v;
}

// Warp-aggregated append of one element per participating lane.  All 32 lanes
// of the warp must call it (converged); lanes with `want` false contribute
// nothing.  Returns the slot index for lanes with want, else undefined.
__device__ __forceinline__ uint32_t warp_append_slot(bool want, uint32_t *counter) {
    const uint32_t mask = __ballot_sync(0xffffffffu, want);
    uint32_t base = 0;
    if (mask) {
        const int leader = __ffs(mask) - 1;
        if (lane_id() == leader) base = atomicAdd(counter, (uint32_t)__popc(mask));
        base = __shfl_sync(0xffffffffu, base, leader);
    }
    return base + __popc(mask & lanemask_lt());
}

// Warp-aggregated reservation of `cnt` consecutive slots per lane.
__device__ __forceinline__ uint32_t warp_reserve(uint32_t cnt, uint32_t *counter) {
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane_id() >= o) incl += t;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    uint32_t base = 0;
    if (total) {
        if (lane_id() == 31) base = atomicAdd(counter, total);
        base = __shfl_sync(0xffffffffu, base, 31);
    }
    return base + incl - cnt;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------- host helpers

struct DeviceInfo {
    int device = -1;
    int sms = 0;
    int l2_bytes = 0;
    int max_smem_optin = 0;
};

// Queried once per device (cudaGetDevice / cudaDeviceGetAttribute only).
DeviceInfo device_info();

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bump allocator over a caller workspace.
struct Carve {
    char *base;
    size_t off;
    explicit Carve(void *b) : base((char *)b), off(kHeaderBytes) {}
    template <typename T>
    T *take(size_t count) {
        off = align_up(off, 256);
        T *p = (T *)(base ? base + off : nullptr);
        off += count * sizeof(T);
        return p;
    }
    size_t bytes() const { return align_up(off, 256); }
};

inline long long deadline_from(const llp_sched_t *s) {
    return (s && s->deadline_ns > 0) ? s->deadline_ns : kDefaultDeadlineNs;
}

// Launches a cooperative kernel with the largest co-resident grid (capped at
// max_blocks).  Returns LLP_OK or LLP_ERR_CUDA.
llp_status_t launch_cooperative(const void *func, int threads, size_t smem, int max_blocks, void **args,
                                cudaStream_t stream, int *grid_out = nullptr);

llp_status_t reset_header(void *ws, cudaStream_t stream);

}  // namespace llp

#define LLP_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) {                             \
            (void)cudaGetLastError();                        \
            return LLP_ERR_CUDA;                             \
        }                                                    \
    } while (0)

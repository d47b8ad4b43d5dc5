// Transpose of a CSR graph: the in-arc rows that pull sweeps of llp_bfs_pull
// scan.  Input preparation, not a step of the method.
//   1. in-degree histogram (one atomic add per arc; targets outside [0, n)
//      are skipped and reported);
//   2. exclusive scan of the histogram into the new offsets (tile sums, one
//      CTA scans the tile sums, tiles add their prefix) and a copy of the
//      offsets as per-row cursors;
//   3. scatter: each thread walks a run of consecutive arcs (one binary search
//      for the source of its first arc, then forward), and claims a slot of
//      the target's row with an atomic add on its cursor.
// The order within a row follows the order of the atomic adds, so it varies
// from run to run; offsets and the rows as multisets do not.
#include <algorithm>

#include "llp_common.cuh"

namespace llp {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int64_t kScanTile = (int64_t)kScanThreads * kScanItems;
constexpr int kRun = 16;  // arcs per thread in the scatter

__device__ __forceinline__ void atomic_add_off(int32_t *p, int32_t v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add_off(int64_t *p, int64_t v) {
    atomicAdd((unsigned long long *)p, (unsigned long long)v);
}
__device__ __forceinline__ int32_t atomic_take(int32_t *p) { return atomicAdd(p, 1); }
__device__ __forceinline__ int64_t atomic_take(int64_t *p) {
    return (int64_t)atomicAdd((unsigned long long *)p, 1ull);
}

template <typename OffT>
__global__ void tr_count(const int32_t *idx, int64_t m, int32_t n, OffT *cnt, WsHeader *h) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int32_t v = __ldg(idx + e);
        if ((uint32_t)v < (uint32_t)n) {
            atomic_add_off(cnt + v, (OffT)1);
        } else {
            set_status(h, LLP_ERR_INVALID_ARG);
        }
    }
}

// Exclusive scan of one value per thread over the CTA; returns the CTA total.
template <typename T>
__device__ __forceinline__ T cta_exclusive_scan(T x, T &total) {
    __shared__ T s_warp[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        T w = lane < nw ? s_warp[lane] : (T)0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < nw) s_warp[lane] = w;  // inclusive prefix of warp sums
    }
    __syncthreads();
    const T before = wid > 0 ? s_warp[wid - 1] : (T)0;
    total = s_warp[(blockDim.x >> 5) - 1];
    __syncthreads();  // s_warp is reused by the next call
    return before + incl - x;
}

template <typename OffT>
__global__ void __launch_bounds__(kScanThreads) tr_tile_sums(const OffT *cnt, int32_t n, OffT *sums) {
    const int64_t i0 = blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    OffT x = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; j++)
        if (i0 + j < n) x += cnt[i0 + j];
    OffT total;
    (void)cta_exclusive_scan<OffT>(x, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// One CTA: exclusive scan of the tile sums in place; out_off[n] = the total.
template <typename OffT>
__global__ void __launch_bounds__(kScanThreads) tr_scan_sums(OffT *sums, int64_t ntiles, OffT *out_off, int32_t n) {
    OffT carry = 0;
    for (int64_t b = 0; b < ntiles; b += kScanThreads) {
        const int64_t i = b + threadIdx.x;
        const OffT x = i < ntiles ? sums[i] : (OffT)0;
        OffT total;
        const OffT ex = cta_exclusive_scan<OffT>(x, total);
        if (i < ntiles) sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) out_off[n] = carry;
}

template <typename OffT>
__global__ void __launch_bounds__(kScanThreads) tr_scan_tiles(OffT *cnt, int32_t n, const OffT *sums, OffT *out_off) {
    const int64_t i0 = blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    OffT v[kScanItems];
    OffT x = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        v[j] = (i0 + j < n) ? cnt[i0 + j] : (OffT)0;
        x += v[j];
    }
    OffT total;
    OffT run = sums[blockIdx.x] + cta_exclusive_scan<OffT>(x, total);
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        if (i0 + j < n) {
            out_off[i0 + j] = run;
            cnt[i0 + j] = run;  // from here on: the row's cursor
        }
        run += v[j];
    }
}

template <typename OffT>
__global__ void tr_scatter(const OffT *off, const int32_t *idx, const uint32_t *w, int32_t n, int64_t m,
                           OffT *cursor, int32_t *in_idx, uint32_t *in_w) {
    const int64_t runs = (m + kRun - 1) / kRun;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < runs; r += stride) {
        const int64_t e0 = r * kRun;
        const int64_t e1 = min(e0 + (int64_t)kRun, m);
        // source of arc e0: the last u with off[u] <= e0
        int32_t lo = 0, hi = n;  // off[lo] <= e0 < off[hi] (off[n] = m > e0)
        while (hi - lo > 1) {
            const int32_t mid = lo + (hi - lo) / 2;
            if ((int64_t)__ldg(off + mid) <= e0) lo = mid; else hi = mid;
        }
        int32_t u = lo;
        int64_t row_end = (int64_t)__ldg(off + u + 1);
        for (int64_t e = e0; e < e1; e++) {
            while (row_end <= e && u < n - 1) {  // (offsets are non-decreasing with off[n] = m)
                u++;
                row_end = (int64_t)__ldg(off + u + 1);
            }
            const int32_t v = __ldg(idx + e);
            if ((uint32_t)v >= (uint32_t)n) continue;
            const OffT pos = atomic_take(cursor + v);
            in_idx[pos] = u;
            if (in_w) in_w[pos] = __ldg(w + e);
        }
    }
}

struct TrLayout {
    void *cnt;
    void *sums;
    size_t bytes;
};

TrLayout carve_transpose(void *ws, int32_t n, bool off64) {
    Carve c(ws);
    TrLayout L;
    const size_t ntiles = (size_t)(((int64_t)n + kScanTile - 1) / kScanTile);
    if (off64) {
        L.cnt = c.take<int64_t>((size_t)n);
        L.sums = c.take<int64_t>(ntiles + 1);
    } else {
        L.cnt = c.take<int32_t>((size_t)n);
        L.sums = c.take<int32_t>(ntiles + 1);
    }
    L.bytes = c.bytes();
    return L;
}

template <typename OffT>
llp_status_t transpose_impl(const llp_csr_t *g, OffT *out_off, int32_t *in_idx, uint32_t *in_w, const TrLayout &L,
                            void *ws, cudaStream_t st) {
    const int32_t n = g->n;
    const int64_t m = g->m;
    OffT *cnt = (OffT *)L.cnt;
    OffT *sums = (OffT *)L.sums;
    WsHeader *h = (WsHeader *)ws;
    const int64_t ntiles = ((int64_t)n + kScanTile - 1) / kScanTile;
    const int sms = device_info().sms > 0 ? device_info().sms : 148;
    LLP_CUDA_TRY(cudaMemsetAsync(cnt, 0, (size_t)n * sizeof(OffT), st));
    if (m > 0) {
        tr_count<OffT><<<sms * 8, 256, 0, st>>>(g->indices, m, n, cnt, h);
        LLP_CUDA_TRY(cudaGetLastError());
    }
    tr_tile_sums<OffT><<<(unsigned)ntiles, kScanThreads, 0, st>>>(cnt, n, sums);
    LLP_CUDA_TRY(cudaGetLastError());
    tr_scan_sums<OffT><<<1, kScanThreads, 0, st>>>(sums, ntiles, out_off, n);
    LLP_CUDA_TRY(cudaGetLastError());
    tr_scan_tiles<OffT><<<(unsigned)ntiles, kScanThreads, 0, st>>>(cnt, n, sums, out_off);
    LLP_CUDA_TRY(cudaGetLastError());
    if (m > 0) {
        const int64_t runs = (m + kRun - 1) / kRun;
        const int64_t blocks = std::min<int64_t>((runs + 255) / 256, (int64_t)sms * 16);
        tr_scatter<OffT><<<(unsigned)blocks, 256, 0, st>>>((const OffT *)g->offsets, g->indices, in_w ? g->weights : nullptr,
                                                         n, m, cnt, in_idx, in_w);
        LLP_CUDA_TRY(cudaGetLastError());
    }
    return LLP_OK;
}

}  // namespace
}  // namespace llp

extern "C" {

size_t llp_csr_transpose_workspace_size(int32_t n, int64_t m) {
    if (n < 1 || m < 0) return 0;
    return llp::carve_transpose(nullptr, n, true).bytes;
}

llp_status_t llp_csr_transpose(const llp_csr_t *g, void *in_offsets, int32_t *in_indices, uint32_t *in_weights,
                               void *ws, size_t ws_bytes, void *stream) {
    if (!g || !in_offsets || !ws) return LLP_ERR_INVALID_ARG;
    if (g->n < 1 || g->m < 0 || !g->offsets) return LLP_ERR_INVALID_ARG;
    if (g->m > 0 && (!g->indices || !in_indices)) return LLP_ERR_INVALID_ARG;
    if (in_weights && g->m > 0 && !g->weights) return LLP_ERR_INVALID_ARG;
    if (!g->offsets_64 && g->m > 0x7FFFFFFFll) return LLP_ERR_INVALID_ARG;
    if (((uintptr_t)ws & 255u) != 0) return LLP_ERR_INVALID_ARG;
    const llp::TrLayout L = llp::carve_transpose(ws, g->n, g->offsets_64 != 0);
    if (ws_bytes < L.bytes) return LLP_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t st = (cudaStream_t)stream;
    const llp_status_t rc = llp::reset_header(ws, st);
    if (rc != LLP_OK) return rc;
    if (g->offsets_64)
        return llp::transpose_impl<int64_t>(g, (int64_t *)in_offsets, in_indices, in_weights, L, ws, st);
    return llp::transpose_impl<int32_t>(g, (int32_t *)in_offsets, in_indices, in_weights, L, ws, st);
}

}  // extern "C"

// Learned scheduler of the graph sweep (an adaptive choice of solver, which the
// paper leaves to future work in its conclusion): a small MLP
//     16 instance features -> 64 -> 64 -> logits of five softmax heads
//     {sweep mode (3), bucket-width class (8), work-block configuration (3),
//      local-chain class (4: off, 4, 16, 64 batches),
//      dense-sweep group-width class (5: the grid-size rule, 1, 2, 4, 8 words)}
// with ReLU activations, fp32.  It only picks the schedule of a run; the
// schedule never changes the result (every schedule reaches the same least
// fixed point), so a bad choice only costs time.
//
// Kernels here: instance features (one CTA, sampled), inference on one feature
// vector (writes the schedule into the workspace header, read by the sweep
// kernel), and the training path: forward, per-sample backward, per-parameter
// gradient reduction, Adam step.  Parameter layout (row-major, one vector):
//     W1[F,H1] b1[H1] W2[H1,H2] b2[H2] W3[H2,O] b3[O].
#include <math.h>

#include <algorithm>

#include "llp_common.cuh"
#include "sweep_init.cuh"

namespace llp {

constexpr int kMaxDim = 128;

struct MlpDims {
    int F, H1, H2, O;
    int nheads;
    int heads[8];
};

__host__ __device__ inline size_t mlp_param_count(const MlpDims &d) {
    return (size_t)d.F * d.H1 + d.H1 + (size_t)d.H1 * d.H2 + d.H2 + (size_t)d.H2 * d.O + d.O;
}

namespace {

// ------------------------------------------------------------- features

constexpr int kFeatBlocks = 64;
constexpr int kFeatThreads = 256;
constexpr int kFeatSamples = 16384;  // vertices and arcs sampled (evenly spaced)

// Instance features from an evenly spaced sample of vertices (degree
// histogram, mean and max degree) and arcs (weight range and spread).  CTAs
// cta = 0 .. ncta-1 accumulate into the header; the last CTA to finish writes
// the features and returns true (to all its threads).  Every thread of a
// participating CTA calls it.
template <typename OffT>
__device__ bool features_part(int32_t n, int64_t m, const OffT *off, const uint32_t *w, int32_t source, WsHeader *h,
                              int cta, int ncta) {
    __shared__ unsigned int s_hist[6];
    __shared__ unsigned long long s_deg;
    __shared__ unsigned int s_maxdeg, s_wmin, s_wmax;
    __shared__ float s_wsum, s_wsq;
    __shared__ int s_last;
    if (threadIdx.x < 6) s_hist[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        s_deg = 0;
        s_maxdeg = 0;
        s_wmin = 0xFFFFFFFFu;
        s_wmax = 0;
        s_wsum = 0.f;
        s_wsq = 0.f;
    }
    __syncthreads();
    const int32_t S = n < kFeatSamples ? n : kFeatSamples;
    const int64_t Sw = m < kFeatSamples ? m : kFeatSamples;
    const int stride = ncta * blockDim.x;
    unsigned long long dsum = 0;
    unsigned int dmax = 0;
    for (int32_t i = cta * blockDim.x + threadIdx.x; i < S; i += stride) {
        const int64_t v = (int64_t)i * n / S;
        const unsigned int d = (unsigned int)(off[v + 1] - off[v]);
        const int b = d == 0 ? 0 : d < 4 ? 1 : d < 16 ? 2 : d < 64 ? 3 : d < 256 ? 4 : 5;
        atomicAdd(&s_hist[b], 1u);
        dsum += d;
        dmax = max(dmax, d);
    }
    unsigned int wmn = 0xFFFFFFFFu, wmx = 0;
    float ws = 0.f, wq = 0.f;
    for (int64_t i = (int64_t)cta * blockDim.x + threadIdx.x; i < Sw && w; i += stride) {
        const unsigned int x = w[i * m / Sw];
        wmn = min(wmn, x);
        wmx = max(wmx, x);
        ws += (float)x;
        wq += (float)x * (float)x;
    }
    // warp reductions first: one shared-memory atomic per warp and quantity
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
        dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        wmn = min(wmn, __shfl_xor_sync(0xffffffffu, wmn, o));
        wmx = max(wmx, __shfl_xor_sync(0xffffffffu, wmx, o));
        ws += __shfl_xor_sync(0xffffffffu, ws, o);
        wq += __shfl_xor_sync(0xffffffffu, wq, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&s_deg, dsum);
        atomicMax(&s_maxdeg, dmax);
        atomicMin(&s_wmin, wmn);
        atomicMax(&s_wmax, wmx);
        atomicAdd(&s_wsum, ws);
        atomicAdd(&s_wsq, wq);
    }
    __syncthreads();
    // header accumulators: scratch[9..14] (zeroed with the header)
    uint32_t *acc = h->scratch + 9;
    if (threadIdx.x < 6) atomicAdd(acc + threadIdx.x, s_hist[threadIdx.x]);
    if (threadIdx.x == 0) {
        atomicMax((unsigned int *)&h->feat[0], s_maxdeg);  // staged in feat[] bit patterns
        atomicMax((unsigned int *)&h->feat[1], s_wmax);
        atomicMax((unsigned int *)&h->feat[2], ~s_wmin);    // max of complements = min
        atomicAdd(&h->feat[3], s_wsum);
        atomicAdd(&h->feat[4], s_wsq);
        __threadfence();
        s_last = atomicAdd(&h->scratch[15], 1u) + 1u == (unsigned)ncta;
    }
    __syncthreads();
    if (!s_last) return false;
    if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int maxdeg = *(volatile unsigned int *)&h->feat[0];
    const unsigned int swmax = *(volatile unsigned int *)&h->feat[1];
    const unsigned int swmin = ~*(volatile unsigned int *)&h->feat[2];
    const float wsum = *(volatile float *)&h->feat[3], wsq = *(volatile float *)&h->feat[4];
    unsigned int hist[6];
    for (int b = 0; b < 6; b++) hist[b] = *(volatile uint32_t *)&acc[b];
    const float fs = (float)(S > 0 ? S : 1);
    const unsigned int sdeg = (unsigned int)(off[source + 1] - off[source]);
    float *f = h->feat;
    const bool unit = (w == nullptr) || Sw == 0;
    const float wmax = unit ? 1.f : (float)swmax;
    const float wmin = unit ? 1.f : (float)swmin;
    const float mean = unit ? 1.f : wsum / (float)Sw;
    const float var = unit ? 0.f : fmaxf(wsq / (float)Sw - mean * mean, 0.f);
    f[0] = log2f((float)n + 1.f);
    f[1] = log2f((float)m + 1.f);
    f[2] = log2f((float)m / (float)n + 1.f);
    for (int b = 0; b < 6; b++) f[3 + b] = (float)hist[b] / fs;
    f[9] = log2f((float)max(maxdeg, sdeg) + 1.f);
    f[10] = log2f(wmax + 1.f);
    f[11] = log2f(wmin + 1.f);
    f[12] = sqrtf(var) / fmaxf(mean, 1e-6f);
    f[13] = unit ? 1.f : 0.f;
    f[14] = log2f((float)sdeg + 1.f) - f[2];
    f[15] = 1.f;
    h->feat_wmax = wmax;
    __threadfence();
    }
    __syncthreads();
    return true;
}

template <typename OffT>
__global__ void __launch_bounds__(kFeatThreads) graph_features_kernel(int32_t n, int64_t m, const OffT *off,
                                                                      const uint32_t *w, int32_t source, WsHeader *h) {
    features_part(n, m, off, w, source, h, blockIdx.x, gridDim.x);
}

// ------------------------------------------------------------- inference

__device__ __forceinline__ int argmax_head(const float *z, int lo, int len) {
    int best = lo;
    for (int i = lo + 1; i < lo + len; i++)
        if (z[i] > z[best]) best = i;
    return best - lo;
}

// One CTA (>= max(H1, H2, O) threads): MLP on h->feat, then the schedule.
// The parameters are first copied to shared memory (sp, kSchedSmemParams
// floats) with independent loads (the layer loops then read shared memory
// instead of waiting on one global load per step); networks larger than the
// buffer read them in place.  Every thread of the CTA calls it.
constexpr int kSchedSmemParams = 8192;
constexpr int kSchedThreads = 256;  // >= kMaxDim; all threads copy the parameters
// Copies the parameters into sp when they fit; returns the pointer the network reads.
__device__ const float *stage_params(const float *params, const MlpDims &d, float *sp) {
    const int t = threadIdx.x;
    const int np = (int)mlp_param_count(d);
    const float *P = params;
    if (np <= kSchedSmemParams) {
        constexpr int U = 8;  // independent loads in flight per thread
        for (int i0 = t; i0 < np; i0 += U * blockDim.x) {
            float r[U];
#pragma unroll
            for (int j = 0; j < U; j++) {
                const int i = i0 + j * blockDim.x;
                r[j] = i < np ? __ldg(params + i) : 0.f;
            }
#pragma unroll
            for (int j = 0; j < U; j++) {
                const int i = i0 + j * blockDim.x;
                if (i < np) sp[i] = r[j];
            }
        }
        P = sp;
    }
    return P;
}

// The network on h->feat with parameters P (shared or global memory), then the schedule.
__device__ void mlp_infer_header(const float *P, const MlpDims &d, WsHeader *h) {
    __shared__ float x[kMaxDim], h1[kMaxDim], h2[kMaxDim], z[kMaxDim];
    const int t = threadIdx.x;
    const float *W1 = P, *b1 = W1 + d.F * d.H1, *W2 = b1 + d.H1, *b2 = W2 + d.H1 * d.H2, *W3 = b2 + d.H2,
                *b3 = W3 + d.H2 * d.O;
    if (t < d.F) x[t] = h->feat[t];
    __syncthreads();
    if (t < d.H1) {
        float a = b1[t];
        for (int i = 0; i < d.F; i++) a = fmaf(x[i], W1[i * d.H1 + t], a);
        h1[t] = fmaxf(a, 0.f);
    }
    __syncthreads();
    if (t < d.H2) {
        float a = b2[t];
        for (int i = 0; i < d.H1; i++) a = fmaf(h1[i], W2[i * d.H2 + t], a);
        h2[t] = fmaxf(a, 0.f);
    }
    __syncthreads();
    if (t < d.O) {
        float a = b3[t];
        for (int i = 0; i < d.H2; i++) a = fmaf(h2[i], W3[i * d.O + t], a);
        z[t] = a;
    }
    __syncthreads();
    if (t == 0) {
        const int mode = argmax_head(z, 0, d.heads[0]);
        const int dc = argmax_head(z, d.heads[0], d.heads[1]);
        const int cfg = argmax_head(z, d.heads[0] + d.heads[1], d.heads[2]);
        h->sched_mode = mode;  // LLP_MODE_AUTO / SPARSE / DENSE
        uint32_t delta = kInf;
        if (dc > 0) {          // class c >= 1: width = wmax * 2^(c-1), at least 1
            const float wd = ldexpf(h->feat_wmax, dc - 1);
            delta = wd < 1.f ? 1u : (wd > 2147483647.f ? 2147483647u : (uint32_t)wd);
        }
        h->sched_delta = delta;
        h->sched_cfg = cfg + 1;
        h->sched_chain = 0;
        if (d.nheads > 3) {
            const int ch = argmax_head(z, d.heads[0] + d.heads[1] + d.heads[2], d.heads[3]);
            h->sched_chain = ch == 0 ? 0 : (1 << (2 * ch));  // 0, 4, 16, 64
        }
        h->sched_gw = 0;
        if (d.nheads > 4) {
            const int gc = argmax_head(z, d.heads[0] + d.heads[1] + d.heads[2] + d.heads[3], d.heads[4]);
            h->sched_gw = gc == 0 ? 0 : (1 << (gc - 1));  // rule, 1, 2, 4, 8
        }
        h->sched_valid = 1;
    }
}

__global__ void mlp_schedule_kernel(const float *params, MlpDims d, WsHeader *h) {
    __shared__ float sp[kSchedSmemParams];
    const float *P = stage_params(params, d, sp);
    mlp_infer_header(P, d, h);
}

// The learned scheduler's prologue of a graph sweep: CTAs 0 .. kFeatBlocks-1
// sample the instance, the last of them runs the network; every other CTA
// initialises the sweep's state meanwhile (so a learned run pays for the
// schedule inside the time the initialisation takes anyway).
template <typename OffT>
__global__ void __launch_bounds__(kFeatThreads) learned_prologue_kernel(int32_t n, int64_t m, const OffT *off,
                                                                        const uint32_t *w, int32_t source,
                                                                        WsHeader *h, const float *params, MlpDims d,
                                                                        SweepInit<OffT> init) {
    __shared__ float sp[kSchedSmemParams];
    if (blockIdx.x < kFeatBlocks) {
        // the parameters are staged while sampling (whichever CTA finishes last runs the network)
        const float *P = stage_params(params, d, sp);
        if (features_part(n, m, off, w, source, h, blockIdx.x, kFeatBlocks)) mlp_infer_header(P, d, h);
    } else {
        const int wpb = blockDim.x >> 5;
        sweep_init(init, (int64_t)(blockIdx.x - kFeatBlocks) * wpb + (threadIdx.x >> 5),
                   (int64_t)(gridDim.x - kFeatBlocks) * wpb);
    }
}

// ------------------------------------------------------------- training

// One CTA per sample: forward, softmax cross-entropy over the heads, and the
// per-sample deltas; stores h1, h2 and the deltas for the weight gradients.
__global__ void mlp_backward_sample_kernel(const float *params, MlpDims d, const float *X, const int32_t *Y,
                                           int32_t B, float *buf_h1, float *buf_h2, float *buf_da1,
                                           float *buf_da2, float *buf_dz, float *loss, float *logits) {
    __shared__ float x[kMaxDim], a1[kMaxDim], h1[kMaxDim], a2[kMaxDim], h2[kMaxDim], z[kMaxDim], dz[kMaxDim],
        da2[kMaxDim];
    const float *W1 = params, *b1 = W1 + d.F * d.H1, *W2 = b1 + d.H1, *b2 = W2 + d.H1 * d.H2, *W3 = b2 + d.H2,
                *b3 = W3 + d.H2 * d.O;
    const int b = blockIdx.x, t = threadIdx.x;
    if (t < d.F) x[t] = X[(size_t)b * d.F + t];
    __syncthreads();
    if (t < d.H1) {
        float a = b1[t];
        for (int i = 0; i < d.F; i++) a = fmaf(x[i], W1[i * d.H1 + t], a);
        a1[t] = a;
        h1[t] = fmaxf(a, 0.f);
    }
    __syncthreads();
    if (t < d.H2) {
        float a = b2[t];
        for (int i = 0; i < d.H1; i++) a = fmaf(h1[i], W2[i * d.H2 + t], a);
        a2[t] = a;
        h2[t] = fmaxf(a, 0.f);
    }
    __syncthreads();
    if (t < d.O) {
        float a = b3[t];
        for (int i = 0; i < d.H2; i++) a = fmaf(h2[i], W3[i * d.O + t], a);
        z[t] = a;
        if (logits) logits[(size_t)b * d.O + t] = a;
    }
    __syncthreads();
    if (t == 0 && Y) {
        float L = 0.f;
        int lo = 0;
        for (int k = 0; k < d.nheads; k++) {
            const int len = d.heads[k];
            float mx = z[lo];
            for (int i = lo + 1; i < lo + len; i++) mx = fmaxf(mx, z[i]);
            float se = 0.f;
            for (int i = lo; i < lo + len; i++) se += expf(z[i] - mx);
            const int y = Y[(size_t)b * d.nheads + k];
            if (y < 0 || y >= len) {  // label outside the head: this head contributes nothing
                for (int i = lo; i < lo + len; i++) dz[i] = 0.f;
                lo += len;
                continue;
            }
            L += logf(se) + mx - z[lo + y];
            for (int i = lo; i < lo + len; i++) dz[i] = (expf(z[i] - mx) / se - (i - lo == y ? 1.f : 0.f)) / B;
            lo += len;
        }
        atomicAdd(loss, L / B);
    }
    if (!Y) return;
    __syncthreads();
    if (t < d.H2) {
        float g = 0.f;
        for (int o = 0; o < d.O; o++) g = fmaf(dz[o], W3[t * d.O + o], g);
        da2[t] = a2[t] > 0.f ? g : 0.f;
    }
    __syncthreads();
    if (t < d.H1) {
        float g = 0.f;
        for (int j = 0; j < d.H2; j++) g = fmaf(da2[j], W2[t * d.H2 + j], g);
        buf_da1[(size_t)b * d.H1 + t] = a1[t] > 0.f ? g : 0.f;
        buf_h1[(size_t)b * d.H1 + t] = h1[t];
    }
    if (t < d.H2) {
        buf_da2[(size_t)b * d.H2 + t] = da2[t];
        buf_h2[(size_t)b * d.H2 + t] = h2[t];
    }
    if (t < d.O) buf_dz[(size_t)b * d.O + t] = dz[t];
}

// One thread per parameter: sum over the batch in a fixed order (deterministic).
__global__ void mlp_grad_reduce_kernel(MlpDims d, const float *X, int32_t B, const float *buf_h1,
                                       const float *buf_h2, const float *buf_da1, const float *buf_da2,
                                       const float *buf_dz, float *grad) {
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nW1 = (size_t)d.F * d.H1, nW2 = (size_t)d.H1 * d.H2, nW3 = (size_t)d.H2 * d.O;
    const size_t o_b1 = nW1, o_W2 = o_b1 + d.H1, o_b2 = o_W2 + nW2, o_W3 = o_b2 + d.H2, o_b3 = o_W3 + nW3,
                 total = o_b3 + d.O;
    if (p >= total) return;
    float g = 0.f;
    if (p < o_b1) {
        const int i = (int)(p / d.H1), j = (int)(p % d.H1);
        for (int b = 0; b < B; b++) g = fmaf(X[(size_t)b * d.F + i], buf_da1[(size_t)b * d.H1 + j], g);
    } else if (p < o_W2) {
        const int j = (int)(p - o_b1);
        for (int b = 0; b < B; b++) g += buf_da1[(size_t)b * d.H1 + j];
    } else if (p < o_b2) {
        const size_t q = p - o_W2;
        const int i = (int)(q / d.H2), j = (int)(q % d.H2);
        for (int b = 0; b < B; b++) g = fmaf(buf_h1[(size_t)b * d.H1 + i], buf_da2[(size_t)b * d.H2 + j], g);
    } else if (p < o_W3) {
        const int j = (int)(p - o_b2);
        for (int b = 0; b < B; b++) g += buf_da2[(size_t)b * d.H2 + j];
    } else if (p < o_b3) {
        const size_t q = p - o_W3;
        const int i = (int)(q / d.O), j = (int)(q % d.O);
        for (int b = 0; b < B; b++) g = fmaf(buf_h2[(size_t)b * d.H2 + i], buf_dz[(size_t)b * d.O + j], g);
    } else {
        const int j = (int)(p - o_b3);
        for (int b = 0; b < B; b++) g += buf_dz[(size_t)b * d.O + j];
    }
    grad[p] = g;
}

// Adam (Kingma and Ba 2015), bias-corrected with step t >= 1.
__global__ void adam_kernel(float *params, const float *grad, float *m, float *v, size_t n, int t, float lr,
                            float b1, float b2, float eps) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - powf(b1, (float)t));
    const float vh = vi / (1.f - powf(b2, (float)t));
    params[i] -= lr * mh / (sqrtf(vh) + eps);
}

bool dims_ok(const MlpDims &d) {
    if (d.F < 1 || d.H1 < 1 || d.H2 < 1 || d.O < 1 || d.F > kMaxDim || d.H1 > kMaxDim || d.H2 > kMaxDim ||
        d.O > kMaxDim || d.nheads < 1 || d.nheads > 8)
        return false;
    int s = 0;
    for (int k = 0; k < d.nheads; k++) {
        if (d.heads[k] < 1) return false;
        s += d.heads[k];
    }
    return s == d.O;
}

MlpDims make_dims(const llp_mlp_dims_t *u) {
    MlpDims d{};
    d.F = u->F;
    d.H1 = u->H1;
    d.H2 = u->H2;
    d.O = u->O;
    d.nheads = u->nheads;
    for (int k = 0; k < 8; k++) d.heads[k] = u->heads[k];
    return d;
}

int block_for(const MlpDims &d) {
    int t = std::max(std::max(d.F, d.H1), std::max(d.H2, d.O));
    return (t + 31) / 32 * 32;
}

}  // namespace

// Used by the graph engine: features + inference for the run about to start.
llp_status_t enqueue_learned_schedule(const llp_csr_t *g, int32_t source, bool unit, const float *params,
                                      WsHeader *h, cudaStream_t st) {
    MlpDims d{};
    d.F = 16;
    d.H1 = 64;
    d.H2 = 64;
    d.O = 23;
    d.nheads = 5;
    d.heads[0] = 3;
    d.heads[1] = 8;
    d.heads[2] = 3;
    d.heads[3] = 4;
    d.heads[4] = 5;
    const uint32_t *w = unit ? nullptr : g->weights;
    if (g->offsets_64)
        graph_features_kernel<int64_t><<<kFeatBlocks, kFeatThreads, 0, st>>>(g->n, g->m, (const int64_t *)g->offsets,
                                                                              w, source, h);
    else
        graph_features_kernel<int32_t><<<kFeatBlocks, kFeatThreads, 0, st>>>(g->n, g->m, (const int32_t *)g->offsets,
                                                                              w, source, h);
    mlp_schedule_kernel<<<1, kSchedThreads, 0, st>>>(params, d, h);
    LLP_CUDA_TRY(cudaGetLastError());
    return LLP_OK;
}

// The prologue launch of a learned graph sweep (features + network + state initialisation).
template <typename OffT>
llp_status_t enqueue_learned_prologue(const llp_csr_t *g, int32_t source, bool unit, const float *params, WsHeader *h,
                                      const SweepInit<OffT> &init, cudaStream_t st) {
    MlpDims d{};
    d.F = 16;
    d.H1 = 64;
    d.H2 = 64;
    d.O = 23;
    d.nheads = 5;
    d.heads[0] = 3;
    d.heads[1] = 8;
    d.heads[2] = 3;
    d.heads[3] = 4;
    d.heads[4] = 5;
    const DeviceInfo di = device_info();
    const int init_ctas = std::max(1, (di.sms > 0 ? di.sms : 148) * 6 - kFeatBlocks);
    learned_prologue_kernel<OffT><<<kFeatBlocks + init_ctas, kFeatThreads, 0, st>>>(
        g->n, g->m, (const OffT *)g->offsets, unit ? nullptr : g->weights, source, h, params, d, init);
    LLP_CUDA_TRY(cudaGetLastError());
    return LLP_OK;
}
template llp_status_t enqueue_learned_prologue<int32_t>(const llp_csr_t *, int32_t, bool, const float *, WsHeader *,
                                                        const SweepInit<int32_t> &, cudaStream_t);
template llp_status_t enqueue_learned_prologue<int64_t>(const llp_csr_t *, int32_t, bool, const float *, WsHeader *,
                                                        const SweepInit<int64_t> &, cudaStream_t);

}  // namespace llp

extern "C" {

size_t llp_mlp_param_count(const llp_mlp_dims_t *dims) {
    if (!dims) return 0;
    return llp::mlp_param_count(llp::make_dims(dims));
}

size_t llp_mlp_workspace_size(const llp_mlp_dims_t *dims, int32_t batch) {
    if (!dims || batch < 0) return 0;
    const llp::MlpDims d = llp::make_dims(dims);
    return llp::kHeaderBytes + (size_t)batch * (2 * d.H1 + 2 * d.H2 + d.O) * 4 + 1024;
}

llp_status_t llp_mlp_forward(const llp_mlp_dims_t *dims, const float *params, const float *X, int32_t batch,
                             float *logits, void *stream) {
    using namespace llp;
    if (!dims || !params || !X || !logits || batch < 0) return LLP_ERR_INVALID_ARG;
    const MlpDims d = make_dims(dims);
    if (!dims_ok(d)) return LLP_ERR_INVALID_ARG;
    if (batch == 0) return LLP_OK;
    mlp_backward_sample_kernel<<<batch, block_for(d), 0, (cudaStream_t)stream>>>(
        params, d, X, nullptr, batch, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, logits);
    LLP_CUDA_TRY(cudaGetLastError());
    return LLP_OK;
}

llp_status_t llp_mlp_loss_grad(const llp_mlp_dims_t *dims, const float *params, const float *X, const int32_t *Y,
                               int32_t batch, float *loss, float *grad, void *ws, size_t ws_bytes, void *stream) {
    using namespace llp;
    if (!dims || !params || !X || !Y || !loss || !grad || !ws || batch < 1) return LLP_ERR_INVALID_ARG;
    const MlpDims d = make_dims(dims);
    if (!dims_ok(d)) return LLP_ERR_INVALID_ARG;
    if (ws_bytes < llp_mlp_workspace_size(dims, batch)) return LLP_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t st = (cudaStream_t)stream;
    float *buf = (float *)((char *)ws + kHeaderBytes);
    float *h1 = buf, *h2 = h1 + (size_t)batch * d.H1, *da1 = h2 + (size_t)batch * d.H2,
          *da2 = da1 + (size_t)batch * d.H1, *dz = da2 + (size_t)batch * d.H2;
    LLP_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(float), st));
    mlp_backward_sample_kernel<<<batch, block_for(d), 0, st>>>(params, d, X, Y, batch, h1, h2, da1, da2, dz, loss,
                                                               nullptr);
    const size_t np = mlp_param_count(d);
    mlp_grad_reduce_kernel<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(d, X, batch, h1, h2, da1, da2, dz, grad);
    LLP_CUDA_TRY(cudaGetLastError());
    return LLP_OK;
}

llp_status_t llp_mlp_adam(float *params, const float *grad, float *m, float *v, size_t n, int32_t step, float lr,
                          float beta1, float beta2, float eps, void *stream) {
    using namespace llp;
    if (!params || !grad || !m || !v || step < 1) return LLP_ERR_INVALID_ARG;
    if (n == 0) return LLP_OK;
    adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, n, step, lr,
                                                                               beta1, beta2, eps);
    LLP_CUDA_TRY(cudaGetLastError());
    return LLP_OK;
}

llp_status_t llp_graph_schedule(const llp_csr_t *g, int32_t source, int32_t unit_weights, const float *params,
                                void *ws, size_t ws_bytes, void *stream, llp_sched_t *h_chosen, float *h_features) {
    using namespace llp;
    if (!g || !params || !ws || g->n < 1 || source < 0 || source >= g->n) return LLP_ERR_INVALID_ARG;
    if (ws_bytes < kHeaderBytes) return LLP_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t st = (cudaStream_t)stream;
    llp_status_t rc = reset_header(ws, st);
    if (rc != LLP_OK) return rc;
    WsHeader *h = (WsHeader *)ws;
    rc = enqueue_learned_schedule(g, source, unit_weights != 0, params, h, st);
    if (rc != LLP_OK) return rc;
    if (h_chosen || h_features) {
        WsHeader hh;
        LLP_CUDA_TRY(cudaStreamSynchronize(st));
        LLP_CUDA_TRY(cudaMemcpy(&hh, ws, sizeof(hh), cudaMemcpyDeviceToHost));
        if (h_chosen) {
            *h_chosen = llp_sched_t{};
            h_chosen->mode = hh.sched_mode;
            h_chosen->delta = hh.sched_delta;
            h_chosen->block_cfg = hh.sched_cfg;
            h_chosen->local_chain = hh.sched_chain;
            h_chosen->group_words = hh.sched_gw;
        }
        if (h_features)
            for (int i = 0; i < 16; i++) h_features[i] = hh.feat[i];
    }
    return LLP_OK;
}

}  // extern "C"

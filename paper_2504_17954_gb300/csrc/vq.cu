// Vector-quantised attribute storage (Sec. 4.4): per basic model, every attribute except the
// mean and the normal gets a scalar codebook shared by all of its components (k-means over the
// model's values of that attribute), and every Gaussian stores one uint8 index per component.
//
// Codebooks from Lloyd's algorithm in one dimension, all (model, attribute) pairs at once:
//   init:   k centroids spaced evenly over [min, max] of the values, c_j = lo + (hi - lo)(j + 0.5)/k;
//   assign: each value goes to its nearest centroid (binary search between consecutive
//           midpoints of the sorted centroids; a value on a midpoint goes to the lower one);
//   update: c_j = mean of its values, formed as c_j + mean(v - c_j) (float32 partial sums of the
//           offsets per chunk, float64 totals), so that a tight or constant cluster keeps its
//           precision; an empty cluster keeps its centroid; order is restored by a running maximum.
// In one dimension the centroids stay sorted, which is what the binary search needs.
#include "common.cuh"

namespace ivrgs {

constexpr int kVqThreads = 256;
constexpr int kVqChunk = 8192;  // Gaussians per block: one model's accumulators in shared memory
constexpr int kVqComps = 15;    // 3 log_scale, 4 quat, 1 opacity_logit, 3 dcolor, 4 kads

__device__ __forceinline__ int vq_attr_of(int comp) {  // component -> codebook
    return comp < 3 ? 0 : comp < 7 ? 1 : comp < 8 ? 2 : comp < 11 ? 3 : 4 + (comp - 11);
}

__device__ __forceinline__ float vq_comp(const ivrgs_gaussians& g, long long i, int comp) {
    const float* ls = static_cast<const float*>(g.log_scale);
    const float* q = static_cast<const float*>(g.quat);
    const float* o = static_cast<const float*>(g.opacity_logit);
    const float* dc = static_cast<const float*>(g.dcolor);
    const float* k = static_cast<const float*>(g.kads);
    if (comp < 3) return ls[3 * i + comp];
    if (comp < 7) return q[4 * i + comp - 3];
    if (comp < 8) return o[i];
    if (comp < 11) return dc[3 * i + comp - 8];
    return k[4 * i + comp - 11];
}

// order-preserving float <-> uint32 (for atomic min / max)
__device__ __forceinline__ unsigned f2o(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float o2f(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__global__ void __launch_bounds__(kVqThreads) k_vq_minmax(const ivrgs_gaussians g, unsigned* __restrict__ mn,
                                                          unsigned* __restrict__ mx) {
    const long long i = (long long)blockIdx.x * kVqThreads + threadIdx.x;
    const bool active = i < g.n;
    const int m = active ? g.model_id[i] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, m);
    for (int c = 0; c < kVqComps; ++c) {
        const unsigned v = active ? f2o(vq_comp(g, i, c)) : 0u;
        unsigned lo = active ? v : 0xffffffffu, hi = v;
        if (peers == 0xffffffffu) {  // the warp shares a model: one atomic per warp
            lo = __reduce_min_sync(0xffffffffu, lo);
            hi = __reduce_max_sync(0xffffffffu, hi);
            if ((threadIdx.x & 31) == 0 && m >= 0) {
                atomicMin(&mn[m * IVRGS_VQ_ATTRS + vq_attr_of(c)], lo);
                atomicMax(&mx[m * IVRGS_VQ_ATTRS + vq_attr_of(c)], hi);
            }
        } else if (active) {
            atomicMin(&mn[m * IVRGS_VQ_ATTRS + vq_attr_of(c)], lo);
            atomicMax(&mx[m * IVRGS_VQ_ATTRS + vq_attr_of(c)], hi);
        }
    }
}

__global__ void k_vq_init(const unsigned* __restrict__ mn, const unsigned* __restrict__ mx, int n_ma, int K,
                          float* __restrict__ cent) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_ma * K) return;
    const int ma = t / K, j = t % K;
    float lo = o2f(mn[ma]), hi = o2f(mx[ma]);
    if (mn[ma] == 0xffffffffu) lo = hi = 0.0f;  // no Gaussian of this model
    cent[t] = lo + (hi - lo) * ((float)j + 0.5f) / (float)K;
}

// nearest of the sorted centroids c[0..K): the count of midpoints strictly below v
__device__ __forceinline__ int vq_nearest(const float* c, int K, float v) {
    int lo = 0, hi = K - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (v > 0.5f * (c[mid] + c[mid + 1])) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kVqThreads) k_vq_assign(const ivrgs_gaussians g, const float* __restrict__ cent,
                                                          int K, double* __restrict__ sum,
                                                          unsigned* __restrict__ cnt) {
    __shared__ float s_sum[IVRGS_VQ_ATTRS * IVRGS_VQ_MAX_K];
    __shared__ unsigned s_cnt[IVRGS_VQ_ATTRS * IVRGS_VQ_MAX_K];
    const long long c0 = (long long)blockIdx.x * kVqChunk;
    const long long c1 = c0 + kVqChunk < g.n ? c0 + kVqChunk : g.n;
    const int m0 = g.model_id[c0];  // the chunk's first model uses the shared accumulators
    for (int t = threadIdx.x; t < IVRGS_VQ_ATTRS * K; t += kVqThreads) {
        s_sum[t] = 0.0f;
        s_cnt[t] = 0u;
    }
    __syncthreads();
    for (long long i = c0 + threadIdx.x; i < c1; i += kVqThreads) {
        const int m = g.model_id[i];
        for (int c = 0; c < kVqComps; ++c) {
            const int a = vq_attr_of(c);
            const float v = vq_comp(g, i, c);
            const float* cc = cent + ((long long)m * IVRGS_VQ_ATTRS + a) * K;
            const int j = vq_nearest(cc, K, v);
            const float d = v - cc[j];  // offset from the current centroid
            if (m == m0) {
                atomicAdd(&s_sum[a * K + j], d);
                atomicAdd(&s_cnt[a * K + j], 1u);
            } else {
                const long long o = ((long long)m * IVRGS_VQ_ATTRS + a) * K + j;
                atomicAdd(&sum[o], (double)d);
                atomicAdd(&cnt[o], 1u);
            }
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < IVRGS_VQ_ATTRS * K; t += kVqThreads)
        if (s_cnt[t]) {
            const long long o = (long long)m0 * IVRGS_VQ_ATTRS * K + t;
            atomicAdd(&sum[o], (double)s_sum[t]);
            atomicAdd(&cnt[o], s_cnt[t]);
        }
}

// one thread per (model, attribute): means, kept order, accumulators cleared for the next pass
__global__ void k_vq_update(float* __restrict__ cent, double* __restrict__ sum, unsigned* __restrict__ cnt, int n_ma,
                            int K) {
    const int ma = blockIdx.x * blockDim.x + threadIdx.x;
    if (ma >= n_ma) return;
    float* c = cent + (long long)ma * K;
    double* s = sum + (long long)ma * K;
    unsigned* n = cnt + (long long)ma * K;
    float run = -INFINITY;
    for (int j = 0; j < K; ++j) {
        float v = n[j] ? (float)((double)c[j] + s[j] / (double)n[j]) : c[j];
        v = fmaxf(v, run);
        run = v;
        c[j] = v;
        s[j] = 0.0;
        n[j] = 0u;
    }
}

__global__ void __launch_bounds__(kVqThreads) k_vq_encode(const ivrgs_gaussians g, const float* __restrict__ cent,
                                                          int K, const ivrgs_gaussians out) {
    const long long i = (long long)blockIdx.x * kVqThreads + threadIdx.x;
    if (i >= g.n) return;
    const int m = g.model_id[i];
    unsigned char idx[kVqComps];
    for (int c = 0; c < kVqComps; ++c) {
        const int a = vq_attr_of(c);
        idx[c] = (unsigned char)vq_nearest(cent + ((long long)m * IVRGS_VQ_ATTRS + a) * K, K, vq_comp(g, i, c));
    }
    unsigned char* ls = static_cast<unsigned char*>(out.log_scale);
    unsigned char* dc = static_cast<unsigned char*>(out.dcolor);
    for (int k = 0; k < 3; ++k) {
        ls[3 * i + k] = idx[k];
        dc[3 * i + k] = idx[8 + k];
    }
    static_cast<uchar4*>(out.quat)[i] = make_uchar4(idx[3], idx[4], idx[5], idx[6]);
    static_cast<unsigned char*>(out.opacity_logit)[i] = idx[7];
    static_cast<uchar4*>(out.kads)[i] = make_uchar4(idx[11], idx[12], idx[13], idx[14]);
}

size_t vq_workspace(int n_models, int K) {
    const size_t ma = (size_t)n_models * IVRGS_VQ_ATTRS;
    return 256 + ma * 8 + ((ma * K * 4 + 255) & ~size_t(255)) + ma * K * (8 + 4);
}

cudaError_t launch_vq_build(const ivrgs_gaussians* g, int K, int iters, ivrgs_gaussians* out, char* ws,
                            cudaStream_t s) {
    const int n_ma = g->n_models * IVRGS_VQ_ATTRS;
    unsigned* mn = reinterpret_cast<unsigned*>(ws);
    unsigned* mx = mn + n_ma;
    float* cent = reinterpret_cast<float*>(ws + 256 + (size_t)n_ma * 8);
    double* sum = reinterpret_cast<double*>(reinterpret_cast<char*>(cent) + ((((size_t)n_ma * K * 4) + 255) & ~size_t(255)));
    unsigned* cnt = reinterpret_cast<unsigned*>(sum + (size_t)n_ma * K);
    cudaError_t e;
    if ((e = cudaMemsetAsync(mn, 0xff, sizeof(unsigned) * n_ma, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(mx, 0x00, sizeof(unsigned) * n_ma, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(sum, 0, (size_t)n_ma * K * 12, s)) != cudaSuccess) return e;
    IVRGS_PROF("k_vq_build", s);
    const unsigned gb = (unsigned)((g->n + kVqThreads - 1) / kVqThreads);
    if (g->n > 0) k_vq_minmax<<<gb, kVqThreads, 0, s>>>(*g, mn, mx);
    k_vq_init<<<(n_ma * K + 255) / 256, 256, 0, s>>>(mn, mx, n_ma, K, cent);
    const unsigned gc = (unsigned)((g->n + kVqChunk - 1) / kVqChunk);
    for (int it = 0; it < iters && g->n > 0; ++it) {
        k_vq_assign<<<gc, kVqThreads, 0, s>>>(*g, cent, K, sum, cnt);
        k_vq_update<<<(n_ma + 127) / 128, 128, 0, s>>>(cent, sum, cnt, n_ma, K);
    }
    if (g->n > 0) k_vq_encode<<<gb, kVqThreads, 0, s>>>(*g, cent, K, *out);
    if ((e = cudaMemcpyAsync(out->codebook, cent, sizeof(float) * (size_t)n_ma * K, cudaMemcpyDeviceToDevice, s)) !=
        cudaSuccess)
        return e;
    return cudaGetLastError();
}

}  // namespace ivrgs

// Composition, edit table and projection kernels (rows a1, a2 of the path).
#include "gauss_math.cuh"

namespace ivrgs {

// ------------------------------------------------------------------------- composition
struct ModelOffsets {
    int n_models;
    long long off[IVRGS_MAX_MODELS + 1];
};

__global__ void k_model_ids(const __grid_constant__ ModelOffsets mo, uint16_t* __restrict__ model_id, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = mo.n_models - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (mo.off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    model_id[i] = (uint16_t)lo;
}

cudaError_t launch_compose(const ivrgs_gaussians* models, int32_t n_models, ivrgs_gaussians* out, cudaStream_t s) {
    ModelOffsets mo;
    mo.n_models = n_models;
    mo.off[0] = 0;
    for (int m = 0; m < n_models; ++m) mo.off[m + 1] = mo.off[m] + models[m].n;
    for (int m = 0; m < n_models; ++m) {
        const ivrgs_gaussians& src = models[m];
        const long long o = mo.off[m], n = src.n;
        if (n == 0) continue;
        auto F = [](void* p) { return static_cast<float*>(p); };
        const struct { float* d; const void* s; int w; } cp[7] = {
            {F(out->mean) + 3 * o, src.mean, 3},          {F(out->log_scale) + 3 * o, src.log_scale, 3},
            {F(out->quat) + 4 * o, src.quat, 4},          {F(out->opacity_logit) + o, src.opacity_logit, 1},
            {F(out->dcolor) + 3 * o, src.dcolor, 3},      {F(out->normal) + 3 * o, src.normal, 3},
            {F(out->kads) + 4 * o, src.kads, 4}};
        for (const auto& c : cp) {
            cudaError_t e = cudaMemcpyAsync(c.d, c.s, sizeof(float) * c.w * n, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return e;
        }
    }
    const long long n = mo.off[n_models];
    if (n > 0) {
        IVRGS_PROF("k_model_ids", s);
        k_model_ids<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(mo, out->model_id, n);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------- edit table
struct EditParams {
    int n_models;
    float lam[4], bias[4], light[4];
    float e[IVRGS_MAX_MODELS][5];
};

__global__ void k_edit_table(const __grid_constant__ EditParams p, float* __restrict__ table) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int total = p.n_models * IVRGS_EDIT_STRIDE + 12;
    if (i >= total) return;
    float v = 0.0f;
    if (i < p.n_models * IVRGS_EDIT_STRIDE) {
        const int m = i / IVRGS_EDIT_STRIDE, k = i % IVRGS_EDIT_STRIDE;
        v = k < 5 ? p.e[m][k] : 0.0f;
    } else {
        const int k = i - p.n_models * IVRGS_EDIT_STRIDE;
        v = k < 4 ? p.lam[k] : (k < 8 ? p.bias[k - 4] : p.light[k - 8]);
    }
    table[i] = v;
}

cudaError_t launch_edit_table(const ivrgs_model_edit* edits, int32_t n_models, const ivrgs_light* light,
                              float* table, cudaStream_t s) {
    EditParams p;
    p.n_models = n_models;
    for (int k = 0; k < 4; ++k) {
        p.lam[k] = light->lambda[k];
        p.bias[k] = light->bias[k];
    }
    for (int k = 0; k < 3; ++k) p.light[k] = light->dir[k];
    p.light[3] = light->dir_on ? 1.0f : 0.0f;
    for (int m = 0; m < n_models; ++m) {
        p.e[m][0] = edits[m].palette[0];
        p.e[m][1] = edits[m].palette[1];
        p.e[m][2] = edits[m].palette[2];
        p.e[m][3] = edits[m].opacity_scale;
        p.e[m][4] = edits[m].visible ? 1.0f : 0.0f;
    }
    const int total = n_models * IVRGS_EDIT_STRIDE + 12;
    {
        IVRGS_PROF("k_edit_table", s);
        k_edit_table<<<(total + 255) / 256, 256, 0, s>>>(p, table);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------- projection
// One thread per Gaussian: attributes are read once (coalesced structure-of-arrays loads),
// then every view is projected from registers and one record per (view, Gaussian) is written.
template <int PREC>
__global__ void __launch_bounds__(256) k_project(const ivrgs_gaussians g, const float* __restrict__ table,
                                                 const __grid_constant__ CamBatch cb, float lowpass,
                                                 const ivrgs_projected out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = g.n;
    if (i >= n) return;
    GaussLocal G;
    load_gauss<PREC>(g, table, g.n_models, i, G);
    for (int v = 0; v < cb.n; ++v) {
        const long long o = (long long)v * n + i;
        ViewLocal V;
        if (G.visible) project_view(G, cb.c[v], lowpass, V);
        else V.visible = false;
        if (!V.visible) {
            out.radius[o] = 0;
            continue;
        }
        reinterpret_cast<float2*>(out.xy)[o] = make_float2(V.u, V.v);
        reinterpret_cast<float4*>(out.conic_o)[o] = make_float4(V.gam, V.conic[1], V.conic[2], G.o);
        reinterpret_cast<float4*>(out.rgbd)[o] = make_float4(V.rgb[0], V.rgb[1], V.rgb[2], V.depth);
        out.radius[o] = V.radius;
    }
}

cudaError_t launch_project(const ivrgs_gaussians* g, const float* table, const CamBatch& cb, float lowpass,
                           ivrgs_projected* out, cudaStream_t s) {
    if (g->n == 0) return cudaSuccess;
    {
        IVRGS_PROF("k_project", s);
        if (g->precision == IVRGS_VQ)
            k_project<IVRGS_VQ><<<(unsigned)((g->n + 255) / 256), 256, 0, s>>>(*g, table, cb, lowpass, *out);
        else if (g->precision == IVRGS_MIXED)
            k_project<IVRGS_MIXED><<<(unsigned)((g->n + 255) / 256), 256, 0, s>>>(*g, table, cb, lowpass, *out);
        else
            k_project<IVRGS_FP32><<<(unsigned)((g->n + 255) / 256), 256, 0, s>>>(*g, table, cb, lowpass, *out);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------- mixed storage
__device__ __forceinline__ unsigned spread10(unsigned x) {  // 10 bits -> every third bit of 30
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__global__ void k_morton(const float* __restrict__ mean, const uint16_t* __restrict__ model_id, long long n, float3 lo,
                         float3 inv, unsigned long long* __restrict__ keys) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float m[3] = {mean[3 * i], mean[3 * i + 1], mean[3 * i + 2]};
    const float l[3] = {lo.x, lo.y, lo.z}, s[3] = {inv.x, inv.y, inv.z};
    unsigned c[3];
    for (int k = 0; k < 3; ++k) c[k] = (unsigned)fminf(fmaxf((m[k] - l[k]) * s[k] * 1024.0f, 0.0f), 1023.0f);
    const unsigned code = (spread10(c[0]) << 2) | (spread10(c[1]) << 1) | spread10(c[2]);
    keys[i] = ((unsigned long long)model_id[i] << 30) | code;
}

// one CTA per chunk of 256 output Gaussians: gather, anchor at the bounding-box centre, convert
__global__ void __launch_bounds__(IVRGS_ANCHOR_CHUNK) k_pack_mixed(const ivrgs_gaussians in,
                                                                   const unsigned* __restrict__ order,
                                                                   const ivrgs_gaussians out) {
    __shared__ float s_mn[3][IVRGS_ANCHOR_CHUNK / 32], s_mx[3][IVRGS_ANCHOR_CHUNK / 32];
    __shared__ float s_anchor[3];
    const long long n = in.n;
    const long long k = (long long)blockIdx.x * IVRGS_ANCHOR_CHUNK + threadIdx.x;
    const bool valid = k < n;
    const long long src = valid ? (order ? (long long)order[k] : k) : 0;
    const float* im = static_cast<const float*>(in.mean);
    float mu[3] = {0.f, 0.f, 0.f};
    float mn[3], mx[3];
    for (int c = 0; c < 3; ++c) {
        if (valid) mu[c] = im[3 * src + c];
        mn[c] = valid ? mu[c] : INFINITY;
        mx[c] = valid ? mu[c] : -INFINITY;
        for (int o = 16; o > 0; o >>= 1) {
            mn[c] = fminf(mn[c], __shfl_xor_sync(0xffffffffu, mn[c], o));
            mx[c] = fmaxf(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], o));
        }
        if ((threadIdx.x & 31) == 0) {
            s_mn[c][threadIdx.x >> 5] = mn[c];
            s_mx[c][threadIdx.x >> 5] = mx[c];
        }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        float a = INFINITY, b = -INFINITY;
        for (int w = 0; w < IVRGS_ANCHOR_CHUNK / 32; ++w) {
            a = fminf(a, s_mn[threadIdx.x][w]);
            b = fmaxf(b, s_mx[threadIdx.x][w]);
        }
        const float an = __fmul_rn(0.5f, __fadd_rn(a, b));
        s_anchor[threadIdx.x] = an;
        out.anchor[3 * blockIdx.x + threadIdx.x] = an;
    }
    __syncthreads();
    if (!valid) return;
    const float* ls = static_cast<const float*>(in.log_scale);
    const float* dc = static_cast<const float*>(in.dcolor);
    const float* nr = static_cast<const float*>(in.normal);
    __half* om = static_cast<__half*>(out.mean);
    __nv_bfloat16* ols = static_cast<__nv_bfloat16*>(out.log_scale);
    __nv_bfloat16* odc = static_cast<__nv_bfloat16*>(out.dcolor);
    __nv_bfloat16* onr = static_cast<__nv_bfloat16*>(out.normal);
    for (int c = 0; c < 3; ++c) {
        om[3 * k + c] = __float2half_rn(__fsub_rn(mu[c], s_anchor[c]));
        ols[3 * k + c] = __float2bfloat16_rn(ls[3 * src + c]);
        odc[3 * k + c] = __float2bfloat16_rn(dc[3 * src + c]);
        onr[3 * k + c] = __float2bfloat16_rn(nr[3 * src + c]);
    }
    const float4 q = static_cast<const float4*>(in.quat)[src];
    const float4 kk = static_cast<const float4*>(in.kads)[src];
    __half2 q01 = __floats2half2_rn(q.x, q.y), q23 = __floats2half2_rn(q.z, q.w);
    __half2 k01 = __floats2half2_rn(kk.x, kk.y), k23 = __floats2half2_rn(kk.z, kk.w);
    uint2 qb, kb;
    qb.x = *reinterpret_cast<unsigned*>(&q01); qb.y = *reinterpret_cast<unsigned*>(&q23);
    kb.x = *reinterpret_cast<unsigned*>(&k01); kb.y = *reinterpret_cast<unsigned*>(&k23);
    static_cast<uint2*>(out.quat)[k] = qb;
    static_cast<uint2*>(out.kads)[k] = kb;
    static_cast<__half*>(out.opacity_logit)[k] = __float2half_rn(static_cast<const float*>(in.opacity_logit)[src]);
    out.model_id[k] = in.model_id[src];
}

cudaError_t launch_morton(const ivrgs_gaussians* g, const float* lo, const float* hi, uint64_t* keys, cudaStream_t s) {
    if (g->n == 0) return cudaSuccess;
    const float3 l = make_float3(lo[0], lo[1], lo[2]);
    const float3 inv = make_float3(1.0f / (hi[0] - lo[0]), 1.0f / (hi[1] - lo[1]), 1.0f / (hi[2] - lo[2]));
    IVRGS_PROF("k_morton", s);
    k_morton<<<(unsigned)((g->n + 255) / 256), 256, 0, s>>>(static_cast<const float*>(g->mean), g->model_id, g->n, l,
                                                           inv, reinterpret_cast<unsigned long long*>(keys));
    return cudaGetLastError();
}

cudaError_t launch_pack_mixed(const ivrgs_gaussians* in, const uint32_t* order, ivrgs_gaussians* out,
                              cudaStream_t s) {
    if (in->n == 0) return cudaSuccess;
    IVRGS_PROF("k_pack_mixed", s);
    k_pack_mixed<<<(unsigned)((in->n + IVRGS_ANCHOR_CHUNK - 1) / IVRGS_ANCHOR_CHUNK), IVRGS_ANCHOR_CHUNK, 0, s>>>(
        *in, order, *out);
    return cudaGetLastError();
}

}  // namespace ivrgs

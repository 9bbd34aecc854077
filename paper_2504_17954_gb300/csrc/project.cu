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
        const struct { float* d; const float* s; int w; } cp[7] = {
            {out->mean + 3 * o, src.mean, 3},          {out->log_scale + 3 * o, src.log_scale, 3},
            {out->quat + 4 * o, src.quat, 4},          {out->opacity_logit + o, src.opacity_logit, 1},
            {out->dcolor + 3 * o, src.dcolor, 3},      {out->normal + 3 * o, src.normal, 3},
            {out->kads + 4 * o, src.kads, 4}};
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
    float lam[4], bias[4];
    float e[IVRGS_MAX_MODELS][5];
};

__global__ void k_edit_table(const __grid_constant__ EditParams p, float* __restrict__ table) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int total = p.n_models * IVRGS_EDIT_STRIDE + 8;
    if (i >= total) return;
    float v = 0.0f;
    if (i < p.n_models * IVRGS_EDIT_STRIDE) {
        const int m = i / IVRGS_EDIT_STRIDE, k = i % IVRGS_EDIT_STRIDE;
        v = k < 5 ? p.e[m][k] : 0.0f;
    } else {
        const int k = i - p.n_models * IVRGS_EDIT_STRIDE;
        v = k < 4 ? p.lam[k] : p.bias[k - 4];
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
    for (int m = 0; m < n_models; ++m) {
        p.e[m][0] = edits[m].palette[0];
        p.e[m][1] = edits[m].palette[1];
        p.e[m][2] = edits[m].palette[2];
        p.e[m][3] = edits[m].opacity_scale;
        p.e[m][4] = edits[m].visible ? 1.0f : 0.0f;
    }
    const int total = n_models * IVRGS_EDIT_STRIDE + 8;
    {
        IVRGS_PROF("k_edit_table", s);
        k_edit_table<<<(total + 255) / 256, 256, 0, s>>>(p, table);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------- projection
// One thread per Gaussian: attributes are read once (coalesced structure-of-arrays loads),
// then every view is projected from registers and one record per (view, Gaussian) is written.
__global__ void __launch_bounds__(256) k_project(const ivrgs_gaussians g, const float* __restrict__ table,
                                                 const __grid_constant__ CamBatch cb, float lowpass,
                                                 const ivrgs_projected out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = g.n;
    if (i >= n) return;
    GaussLocal G;
    load_gauss(g, table, g.n_models, i, G);
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
        reinterpret_cast<float4*>(out.conic_o)[o] = make_float4(V.conic[0], V.conic[1], V.conic[2], G.o);
        reinterpret_cast<float4*>(out.rgbd)[o] = make_float4(V.rgb[0], V.rgb[1], V.rgb[2], V.depth);
        out.radius[o] = V.radius;
    }
}

cudaError_t launch_project(const ivrgs_gaussians* g, const float* table, const CamBatch& cb, float lowpass,
                           ivrgs_projected* out, cudaStream_t s) {
    if (g->n == 0) return cudaSuccess;
    {
        IVRGS_PROF("k_project", s);
        k_project<<<(unsigned)((g->n + 255) / 256), 256, 0, s>>>(*g, table, cb, lowpass, *out);
    }
    return cudaGetLastError();
}

}  // namespace ivrgs

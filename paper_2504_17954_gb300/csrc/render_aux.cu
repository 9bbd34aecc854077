// Auxiliary maps (Sec. 4.2 first equation: depth and normal maps D, N = sum_i T_i alpha_i {d_i, n_i};
// Sec. 4.3: the offset-colour map sum_i T_i alpha_i dc_i and the coefficient maps
// sum_i T_i alpha_i k_i; the attribute render modes of the interface in Sec. 4.7).
//
// The walk is the forward compositing of render.cu at one pixel per thread: the same staged
// thresholds, the same 4-row exponent groups and the same transmittance updates, so every
// pixel has exactly the contributors and weights T_i alpha_i of ivrgs_render (the last output
// channel, 1 - T, equals the alpha of ivrgs_render bit for bit). Each staged entry carries
// its 11 values: camera depth, unit normal (world), offset colour, edited k' = lambda k + b.
#include <type_traits>

#include "blend_alpha.cuh"
#include "gauss_math.cuh"

namespace ivrgs {

constexpr int kAux = 11;

// normal, offset colour and k of Gaussian i in either storage
template <int PREC>
__device__ __forceinline__ void load_aux_attrs(const ivrgs_gaussians& g, long long i, float nrm[3], float dc[3],
                                               float4& kk) {
    if constexpr (PREC == IVRGS_VQ) {
        const int m = g.model_id[i];
        const float* n = static_cast<const float*>(g.normal);
        const unsigned char* ci = static_cast<const unsigned char*>(g.dcolor);
        for (int k = 0; k < 3; ++k) {
            nrm[k] = n[3 * i + k];
            dc[k] = vq_value(g, m, 3, ci[3 * i + k]);
        }
        const uchar4 ki = static_cast<const uchar4*>(g.kads)[i];
        kk = make_float4(vq_value(g, m, 4, ki.x), vq_value(g, m, 5, ki.y), vq_value(g, m, 6, ki.z),
                         vq_value(g, m, 7, ki.w));
    } else if constexpr (PREC == IVRGS_FP32) {
        const float* n = static_cast<const float*>(g.normal);
        const float* c = static_cast<const float*>(g.dcolor);
        for (int k = 0; k < 3; ++k) {
            nrm[k] = n[3 * i + k];
            dc[k] = c[3 * i + k];
        }
        kk = static_cast<const float4*>(g.kads)[i];
    } else {
        const __nv_bfloat16* n = static_cast<const __nv_bfloat16*>(g.normal);
        const __nv_bfloat16* c = static_cast<const __nv_bfloat16*>(g.dcolor);
        for (int k = 0; k < 3; ++k) {
            nrm[k] = __bfloat162float(n[3 * i + k]);
            dc[k] = __bfloat162float(c[3 * i + k]);
        }
        const uint2 kb = static_cast<const uint2*>(g.kads)[i];
        const __half2 k01 = *reinterpret_cast<const __half2*>(&kb.x), k23 = *reinterpret_cast<const __half2*>(&kb.y);
        kk = make_float4(__low2float(k01), __high2float(k01), __low2float(k23), __high2float(k23));
    }
}

template <int PREC, int TH>
__global__ void __launch_bounds__(kTile * TH) k_render_aux(const float2* __restrict__ xy,
                                                         const float4* __restrict__ conic_o,
                                                         const float4* __restrict__ rgbd, long long n,
                                                         const unsigned* __restrict__ values,
                                                         const uint2* __restrict__ ranges,
                                                         const __grid_constant__ CamBatch cb, const ivrgs_gaussians g,
                                                         const float* __restrict__ table, int n_models,
                                                         float4* __restrict__ out) {
    constexpr int kAuxBatch = kTile * TH;  // one staged entry per thread (one pixel each)
    __shared__ float4 s_a[kAuxBatch];
    __shared__ float4 s_b[kAuxBatch];
    __shared__ float2 s_c[kAuxBatch];
    __shared__ float s_x[kAux][kAuxBatch];
    const long long tile = blockIdx.x;
    const int v = view_of_tile(cb, tile);
    const CamDev& cam = cb.c[v];
    const int local = (int)(tile - cam.tile0);
    const int tx = local % cam.gx, ty = local / cam.gx;
    const int px = tx * kTile + (threadIdx.x & (kTile - 1));
    const int py = ty * TH + (int)(threadIdx.x / kTile);
    const float fx = (float)px + 0.5f;
    const int q0 = py & 3;
    const float fyg = (float)(py - q0) + 0.5f;
    const uint2 rg = ranges[tile];
    const long long vbase = (long long)v * n;
    const float* lam = table + (long long)n_models * IVRGS_EDIT_STRIDE;
    const bool inside = px < cam.W && py < cam.H;
    float acc[kAux];
#pragma unroll
    for (int k = 0; k < kAux; ++k) acc[k] = 0.f;
    float T = 1.f;
    bool done = !inside;
    const int len = (int)(rg.y - rg.x);
    for (int b0 = 0; b0 < len; b0 += kAuxBatch) {
        if (__syncthreads_count(done) == kAuxBatch) break;
        {
            const int e = b0 + (int)threadIdx.x;
            if (e < len) {
                const unsigned gg = values[rg.x + e];
                float4 sa, sb;
                float2 sc;
                float x[kAux];
                if (gg < (unsigned long long)n) {
                    const long long gi = vbase + gg;
                    const float4 cd = rgbd[gi];
                    stage_gaussian(xy[gi], conic_o[gi], cd, sa, sb, sc);
                    float nrm[3], dc[3];
                    float4 kk;
                    load_aux_attrs<PREC>(g, gg, nrm, dc, kk);
                    const float il = 1.0f / sqrtf(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
                    const float k4[4] = {kk.x, kk.y, kk.z, kk.w};
                    x[0] = cd.w;
                    for (int k = 0; k < 3; ++k) {
                        x[1 + k] = nrm[k] * il;
                        x[4 + k] = dc[k];
                    }
                    for (int k = 0; k < 4; ++k) x[7 + k] = __ldg(lam + k) * k4[k] + __ldg(lam + 4 + k);
                } else {  // never for a completed sort; a zero-opacity stand-in keeps reads in bounds
                    stage_gaussian(make_float2(0.f, 0.f), make_float4(1.f, 0.f, 1.f, 0.f),
                                   make_float4(0.f, 0.f, 0.f, 0.f), sa, sb, sc);
                    for (int k = 0; k < kAux; ++k) x[k] = 0.f;
                }
                s_a[threadIdx.x] = sa;
                s_b[threadIdx.x] = sb;
                s_c[threadIdx.x] = sc;
#pragma unroll
                for (int k = 0; k < kAux; ++k) s_x[k][threadIdx.x] = x[k];
            }
        }
        __syncthreads();
        if (__all_sync(0xffffffffu, done)) continue;
        const int cnt = min(kAuxBatch, len - b0);
        for (int j = 0; j < cnt; ++j) {
            const float4 a = s_a[j];
            const float4 bb = s_b[j];
            const float2 cc = s_c[j];
            const RowGroup rgp = row_group(a, bb, fx, fyg);
            const float p2 = row_p2(rgp, a, q0);
            const bool ok = !done && in_reach(p2, cc.y);
            if (__any_sync(0xffffffffu, ok)) {
                // the forward blend's update (k_render), so that 1 - T equals its alpha bit for bit
                const float G = fast_ex2(p2);
                const float om =
                    bb.y > kNoClampOpacity ? one_minus_alpha<true>(bb.y, G) : one_minus_alpha<false>(bb.y, G);
                const float Tn = __fmul_rn(T, om);
                const bool stop = ok && Tn < kTMin;
                const bool add = ok && !stop;
                const float Tk = add ? Tn : T;
                const float w = T - Tk;
#pragma unroll
                for (int k = 0; k < kAux; ++k) acc[k] = fmaf(w, s_x[k][j], acc[k]);
                T = Tk;
                done = done || stop;
            }
            if ((j & 7) == 7 && __all_sync(0xffffffffu, done)) break;
        }
    }
    if (inside) {
        float4* o = out + 3 * (cam.pix0 + (long long)py * cam.W + px);
        o[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
        o[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
        o[2] = make_float4(acc[8], acc[9], acc[10], 1.0f - T);
    }
}

cudaError_t launch_render_aux(const ivrgs_gaussians* g, const float* table, const ivrgs_projected* p,
                              const ivrgs_bins* b, const CamBatch& cb, float* aux, cudaStream_t s) {
    if (cb.n_tiles == 0) return cudaSuccess;
    IVRGS_PROF("k_render_aux", s);
    const float2* xy = reinterpret_cast<const float2*>(p->xy);
    const float4* co = reinterpret_cast<const float4*>(p->conic_o);
    const float4* cd = reinterpret_cast<const float4*>(p->rgbd);
    const uint2* rg = reinterpret_cast<const uint2*>(b->ranges);
    float4* out = reinterpret_cast<float4*>(aux);
    auto launch = [&](auto prec) {
        constexpr int kPrec = decltype(prec)::value;
        if (cb.th == 8)
            k_render_aux<kPrec, 8><<<(unsigned)cb.n_tiles, kTile * 8, 0, s>>>(xy, co, cd, p->n, b->values, rg, cb, *g,
                                                                            table, g->n_models, out);
        else
            k_render_aux<kPrec, 16><<<(unsigned)cb.n_tiles, kTile * 16, 0, s>>>(xy, co, cd, p->n, b->values, rg, cb,
                                                                              *g, table, g->n_models, out);
    };
    if (g->precision == IVRGS_VQ) launch(std::integral_constant<int, IVRGS_VQ>{});
    else if (g->precision == IVRGS_MIXED) launch(std::integral_constant<int, IVRGS_MIXED>{});
    else launch(std::integral_constant<int, IVRGS_FP32>{});
    return cudaGetLastError();
}

}  // namespace ivrgs

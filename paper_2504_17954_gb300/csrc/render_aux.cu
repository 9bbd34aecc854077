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

// ---------------------------------------------------------------------------------------------
// Reverse mode of the auxiliary maps. The maps composite each Gaussian's 11 values x_i with the
// weights T_i alpha_i and no background, and the last channel is 1 - T (Sec. 4.2 first
// equation), so the reverse walk is the colour one (k_render_bwd) with x in place of the colour:
// back to front from each pixel's last contributor, T_i = T_{i+1} / (1 - alpha_i) from the stored
// final T, dL/dalpha_i = T_i (dA . x_i) - S_i / (1 - alpha_i) with S the weighted sum behind i
// started at -T_final dL/d(1 - T). Per in-reach (pixel, entry) it adds, with atomics per
// contributing lane, the gradients of the 2D quantities in the layout the projection's reverse
// mode reads (its colour gradient zero) and the 11 value gradients T_i alpha_i dA (record-major,
// 12 floats per record). One pixel per thread, one CTA per tile.
template <int PREC, int TH>
__global__ void __launch_bounds__(kTile * TH) k_render_aux_bwd(
    const float2* __restrict__ xy, const float4* __restrict__ conic_o, const float4* __restrict__ rgbd, long long n,
    const unsigned* __restrict__ values, const uint2* __restrict__ ranges, const __grid_constant__ CamBatch cb,
    const ivrgs_gaussians g, const float* __restrict__ table, int n_models, const float* __restrict__ final_T,
    const unsigned* __restrict__ last_in, const float4* __restrict__ dL, float4* __restrict__ g0,
    float4* __restrict__ g1, float4* __restrict__ gx) {
    constexpr int NB = kTile * TH;  // one staged entry per thread
    __shared__ float4 s_a[NB];
    __shared__ float4 s_b[NB];
    __shared__ float2 s_c[NB];
    __shared__ float s_x[kAux][NB];
    __shared__ long long s_gi[NB];
    __shared__ unsigned s_top;
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
    float T = 1.f, dA[kAux + 1];
    unsigned my_last = 0;
#pragma unroll
    for (int k = 0; k <= kAux; ++k) dA[k] = 0.f;
    if (px < cam.W && py < cam.H) {
        const long long pix = cam.pix0 + (long long)py * cam.W + px;
        T = final_T[pix];
        my_last = last_in[pix];
        const float4 d0 = dL[3 * pix], d1 = dL[3 * pix + 1], d2 = dL[3 * pix + 2];
        dA[0] = d0.x; dA[1] = d0.y; dA[2] = d0.z; dA[3] = d0.w;
        dA[4] = d1.x; dA[5] = d1.y; dA[6] = d1.z; dA[7] = d1.w;
        dA[8] = d2.x; dA[9] = d2.y; dA[10] = d2.z; dA[11] = d2.w;
    }
    float DS = -T * dA[kAux];  // the 1 - T channel: dA/dalpha_i = T_final / (1 - alpha_i)
    if (threadIdx.x == 0) s_top = 0u;
    __syncthreads();
    atomicMax(&s_top, my_last);
    __syncthreads();
    const int top = min((int)s_top, (int)(rg.y - rg.x));
    for (int b_end = top; b_end > 0; b_end -= NB) {
        const int b_start = max(0, b_end - NB);
        __syncthreads();  // the previous batch is walked
        {
            const int e = b_end - 1 - (int)threadIdx.x;  // slot j holds entry b_end - 1 - j
            if (e >= b_start) {
                const unsigned gg = values[rg.x + e];
                float4 sa, sb;
                float2 sc;
                float x[kAux];
                long long gi = -1;
                if (gg < (unsigned long long)n) {
                    gi = vbase + gg;
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
                } else {  // never for a completed sort; a zero-opacity stand-in is never in reach
                    stage_gaussian(make_float2(0.f, 0.f), make_float4(1.f, 0.f, 1.f, 0.f),
                                   make_float4(0.f, 0.f, 0.f, 0.f), sa, sb, sc);
                    for (int k = 0; k < kAux; ++k) x[k] = 0.f;
                }
                s_a[threadIdx.x] = sa;
                s_b[threadIdx.x] = sb;
                s_c[threadIdx.x] = sc;
                s_gi[threadIdx.x] = gi;
#pragma unroll
                for (int k = 0; k < kAux; ++k) s_x[k][threadIdx.x] = x[k];
            }
        }
        __syncthreads();
        const int cnt = b_end - b_start;
        for (int j = 0; j < cnt; ++j) {
            const int e = b_end - 1 - j;
            const float4 a = s_a[j];
            const float4 bb = s_b[j];
            const float2 cc = s_c[j];
            const RowGroup rgp = row_group(a, bb, fx, fyg);
            const float p2 = row_p2(rgp, a, q0);
            const bool ok = e < (int)my_last && in_reach(p2, cc.y);
            if (!__any_sync(0xffffffffu, ok)) continue;
            const float G = fast_ex2(p2);
            const float raw = bb.y * G;
            const float alpha = fminf(kAlphaMax, raw);
            const float r = fast_rcp(1.0f - alpha);
            const float Ti = T * r;
            const float w = ok ? Ti * alpha : 0.0f;
            float dc = 0.f;
#pragma unroll
            for (int k = 0; k < kAux; ++k) dc = fmaf(dA[k], s_x[k][j], dc);
            const float dalpha = Ti * dc - DS * r;
            DS = fmaf(w, dc, DS);
            T = ok ? Ti : T;
            if (ok) {
                // dalpha/dP = o' G below the 0.99 clamp, 0 on it
                const bool live = raw < kAlphaMax;
                const float dP = live ? dalpha * raw : 0.0f;
                const float dop = live ? dalpha * G : 0.0f;
                const float dxp = rgp.dx, dyp = rgp.dy0 - (float)q0;
                const float m1 = dP * dxp, m2 = dP * dyp;
                // moments -> (du, dv, da, db, dc) as in the colour walk: p2 = C' (dy + beta dx)^2 + G' dx^2
                const float il = 2.0f / kLog2e;
                const float tm = fmaf(a.w, m1, m2);
                const long long gi = s_gi[j];
                atomicAdd(g0 + gi, make_float4(fmaf(bb.x, m1, a.z * a.w * tm) * il, a.z * tm * il, -0.5f * m1 * dxp,
                                               -m1 * dyp));
                atomicAdd(g1 + gi, make_float4(-0.5f * m2 * dyp, dop, 0.f, 0.f));
                float4* q = gx + 3 * gi;
                atomicAdd(q, make_float4(w * dA[0], w * dA[1], w * dA[2], w * dA[3]));
                atomicAdd(q + 1, make_float4(w * dA[4], w * dA[5], w * dA[6], w * dA[7]));
                atomicAdd(q + 2, make_float4(w * dA[8], w * dA[9], w * dA[10], 0.f));
            }
        }
    }
}

__device__ __forceinline__ float aux_warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// The value gradients to the stored attributes, summed over the views, added to grad: the camera
// depth z = (R mu + t)_z to the mean (row 2 of R), the unit normal n / |n| to n, dc to dc, and
// k' = lambda k + b to k (lambda k'-gradient) and, block-reduced, to lambda and b.
template <int PREC>
__global__ void __launch_bounds__(256) k_aux_attr_bwd(const ivrgs_gaussians g, const float* __restrict__ table,
                                                      const __grid_constant__ CamBatch cb,
                                                      const float4* __restrict__ gx, const ivrgs_gaussians grad,
                                                      float* __restrict__ egrad) {
    __shared__ float s_red[8][8];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = g.n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float* lam = table + (long long)g.n_models * IVRGS_EDIT_STRIDE;
    float dlam[4] = {0.f, 0.f, 0.f, 0.f}, db[4] = {0.f, 0.f, 0.f, 0.f};
    if (i < n) {
        float dmu[3] = {0.f, 0.f, 0.f}, dn[3] = {0.f, 0.f, 0.f}, ddc[3] = {0.f, 0.f, 0.f};
        float dk[4] = {0.f, 0.f, 0.f, 0.f};
        for (int v = 0; v < cb.n; ++v) {
            const float4* q = gx + 3 * ((long long)v * n + i);
            const float4 a = q[0], b = q[1], c = q[2];
            const float* R = cb.c[v].R;
            for (int k = 0; k < 3; ++k) dmu[k] = fmaf(a.x, R[6 + k], dmu[k]);
            dn[0] += a.y; dn[1] += a.z; dn[2] += a.w;
            ddc[0] += b.x; ddc[1] += b.y; ddc[2] += b.z;
            dk[0] += b.w; dk[1] += c.x; dk[2] += c.y; dk[3] += c.z;
        }
        float nrm[3], dcv[3];
        float4 kk;
        load_aux_attrs<PREC>(g, i, nrm, dcv, kk);
        const float len = sqrtf(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
        const float il = 1.0f / len;
        const float nh[3] = {nrm[0] * il, nrm[1] * il, nrm[2] * il};
        const float dot = nh[0] * dn[0] + nh[1] * dn[1] + nh[2] * dn[2];
        float* gmn = static_cast<float*>(grad.mean);
        float* gno = static_cast<float*>(grad.normal);
        float* gco = static_cast<float*>(grad.dcolor);
        float4* gka = static_cast<float4*>(grad.kads);
        const bool has_dn = dn[0] != 0.f || dn[1] != 0.f || dn[2] != 0.f;  // (no term for an unseen one)
        for (int k = 0; k < 3; ++k) {
            gmn[3 * i + k] += dmu[k];
            if (has_dn) gno[3 * i + k] += (dn[k] - nh[k] * dot) * il;
            gco[3 * i + k] += ddc[k];
        }
        const float k4[4] = {kk.x, kk.y, kk.z, kk.w};
        float4 gk = gka[i];
        gk.x += __ldg(lam + 0) * dk[0];
        gk.y += __ldg(lam + 1) * dk[1];
        gk.z += __ldg(lam + 2) * dk[2];
        gk.w += __ldg(lam + 3) * dk[3];
        gka[i] = gk;
        for (int k = 0; k < 4; ++k) {
            dlam[k] = k4[k] * dk[k];
            db[k] = dk[k];
        }
    }
    float r[8];
    for (int k = 0; k < 4; ++k) {
        r[k] = aux_warp_sum(dlam[k]);
        r[4 + k] = aux_warp_sum(db[k]);
    }
    if (lane == 0)
        for (int k = 0; k < 8; ++k) s_red[warp][k] = r[k];
    __syncthreads();
    if (threadIdx.x < 8) {
        float t = 0.f;
        for (int w = 0; w < 8; ++w) t += s_red[w][threadIdx.x];
        if (t != 0.f) atomicAdd(&egrad[(long long)g.n_models * IVRGS_EDIT_STRIDE + threadIdx.x], t);
    }
}

size_t aux_backward_workspace(long long n, int n_views) {
    const size_t vn = (size_t)n * (size_t)n_views;
    return ((vn * 36 + 15) / 16) * 16 + vn * 48 + 256;
}

cudaError_t launch_render_aux_backward(const ivrgs_gaussians* g, const float* table, const ivrgs_projected* p,
                                       const ivrgs_bins* b, const CamBatch& cb, float lowpass, const float* final_T,
                                       const uint32_t* last, const float* dL, char* ws, ivrgs_gaussians* grad,
                                       float* edit_grad, cudaStream_t s) {
    const long long vn = p->n * (long long)cb.n;
    float4* g0 = reinterpret_cast<float4*>(ws);
    float4* g1 = g0 + vn;
    float* g2 = reinterpret_cast<float*>(g1 + vn);
    float4* gx = reinterpret_cast<float4*>(ws + ((vn * 36 + 15) / 16) * 16);
    cudaError_t e;
    if ((e = cudaMemsetAsync(ws, 0, aux_backward_workspace(p->n, cb.n) - 256, s)) != cudaSuccess) return e;
    const long long ne = (long long)g->n_models * IVRGS_EDIT_STRIDE + 12 + 4ll * cb.n;
    if ((e = cudaMemsetAsync(edit_grad, 0, sizeof(float) * (size_t)ne, s)) != cudaSuccess) return e;
    if (cb.n_tiles > 0) {
        IVRGS_PROF("k_render_aux_bwd", s);
        const float2* xy = reinterpret_cast<const float2*>(p->xy);
        const float4* co = reinterpret_cast<const float4*>(p->conic_o);
        const float4* cd = reinterpret_cast<const float4*>(p->rgbd);
        const uint2* rg = reinterpret_cast<const uint2*>(b->ranges);
        const float4* dl = reinterpret_cast<const float4*>(dL);
        auto launch = [&](auto prec) {
            constexpr int kPrec = decltype(prec)::value;
            if (cb.th == 8)
                k_render_aux_bwd<kPrec, 8><<<(unsigned)cb.n_tiles, kTile * 8, 0, s>>>(
                    xy, co, cd, p->n, b->values, rg, cb, *g, table, g->n_models, final_T, last, dl, g0, g1, gx);
            else
                k_render_aux_bwd<kPrec, 16><<<(unsigned)cb.n_tiles, kTile * 16, 0, s>>>(
                    xy, co, cd, p->n, b->values, rg, cb, *g, table, g->n_models, final_T, last, dl, g0, g1, gx);
        };
        if (g->precision == IVRGS_VQ) launch(std::integral_constant<int, IVRGS_VQ>{});
        else if (g->precision == IVRGS_MIXED) launch(std::integral_constant<int, IVRGS_MIXED>{});
        else launch(std::integral_constant<int, IVRGS_FP32>{});
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // the 2D-quantity gradients through the projection (colour gradient zero), then the values'
    if ((e = launch_project_backward(g, table, cb, lowpass, g0, g1, g2, grad, edit_grad, 0, s)) != cudaSuccess)
        return e;
    if (g->n > 0) {
        IVRGS_PROF("k_aux_attr_bwd", s);
        const unsigned nb = (unsigned)((g->n + 255) / 256);
        if (g->precision == IVRGS_VQ) k_aux_attr_bwd<IVRGS_VQ><<<nb, 256, 0, s>>>(*g, table, cb, gx, *grad, edit_grad);
        else if (g->precision == IVRGS_MIXED)
            k_aux_attr_bwd<IVRGS_MIXED><<<nb, 256, 0, s>>>(*g, table, cb, gx, *grad, edit_grad);
        else k_aux_attr_bwd<IVRGS_FP32><<<nb, 256, 0, s>>>(*g, table, cb, gx, *grad, edit_grad);
    }
    return cudaGetLastError();
}

}  // namespace ivrgs

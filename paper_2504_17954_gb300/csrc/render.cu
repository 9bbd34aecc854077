// Per-tile front-to-back compositing (row a5; Sec. 3 second equation).
//
// One CTA per 16x16 tile; each of its 256/P threads owns P vertically adjacent pixels of one
// column, so every Gaussian staged in shared memory is read once per P pixels and the P
// transmittance chains run interleaved; a warp covers a compact band of 32P/16 rows, so a
// Gaussian that misses the band lets the whole warp skip it. The tile's sorted run is walked in batches of 256
// Gaussians: the CTA stages each batch (mean, conic pre-scaled by -log2(e)/2 so that the
// exponent is one FMA chain, opacity, colour), then every pixel walks it. The CTA leaves as
// soon as every pixel has reached T < 1e-4 (barrier count).
#include "blend_alpha.cuh"

namespace ivrgs {

constexpr int kBatch = 256;

template <int P>
__global__ void __launch_bounds__(kTilePix / P) k_render(const float2* __restrict__ xy,
                                                         const float4* __restrict__ conic_o,
                                                         const float4* __restrict__ rgbd, long long n,
                                                         const unsigned* __restrict__ values,
                                                         const uint2* __restrict__ ranges,
                                                         const __grid_constant__ CamBatch cb, float3 bg,
                                                         float4* __restrict__ rgba, float* __restrict__ final_T,
                                                         unsigned* __restrict__ last_out) {
    constexpr int NT = kTilePix / P;
    __shared__ float4 s_a[kBatch];
    __shared__ float4 s_b[kBatch];
    __shared__ float2 s_c[kBatch];
    const long long tile = blockIdx.x;
    const int v = view_of_tile(cb, tile);
    const CamDev& cam = cb.c[v];
    const int local = (int)(tile - cam.tile0);
    const int tx = local % cam.gx, ty = local / cam.gx;
    const int px = tx * kTile + (threadIdx.x & (kTile - 1));
    const int py0 = ty * kTile + (threadIdx.x / kTile) * P;
    const float fx = (float)px + 0.5f;
    const int q0 = py0 & 3;                               // offset of this thread's first row in its group
    const float fyg = (float)(py0 - q0) + 0.5f;            // centre of the group's first row
    constexpr int NG = (P + 3) / 4;                       // 4-row exponent groups a thread spans
    const uint2 rg = ranges[tile];
    const long long vbase = (long long)v * n;

    float C0[P], C1[P], C2[P], T[P];
    unsigned last[P];
    bool done[P], inside[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int py = py0 + p;
        inside[p] = px < cam.W && py < cam.H;
        C0[p] = C1[p] = C2[p] = 0.f;
        T[p] = 1.f;
        last[p] = 0;
        done[p] = !inside[p];
    }
    const int len = (int)(rg.y - rg.x);
    for (int b0 = 0; b0 < len; b0 += kBatch) {
        bool all = true;
#pragma unroll
        for (int p = 0; p < P; ++p) all = all && done[p];
        if (__syncthreads_count(all) == NT) break;
#pragma unroll
        for (int q = 0; q < kBatch / NT; ++q) {
            const int slot = threadIdx.x + q * NT;
            const int e = b0 + slot;
            if (e < len) {
                const unsigned g = values[rg.x + e];
                float4 sa, sb;
                float2 sc;
                if (g < (unsigned long long)n) {
                    const long long gi = vbase + g;
                    stage_gaussian(xy[gi], conic_o[gi], rgbd[gi], sa, sb, sc);
                } else {  // never for a completed sort; a zero-opacity stand-in keeps reads in bounds
                    stage_gaussian(make_float2(0.f, 0.f), make_float4(1.f, 0.f, 1.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f),
                                   sa, sb, sc);
                }
                s_a[slot] = sa;
                s_b[slot] = sb;
                s_c[slot] = sc;
            }
        }
        __syncthreads();
        // the walk below holds warp-wide votes: a warp skips or leaves it only as a whole
        if (__all_sync(0xffffffffu, all)) continue;
        const int cnt = min(kBatch, len - b0);
        for (int j = 0; j < cnt; ++j) {
            const float4 a = s_a[j];
            const float4 bb = s_b[j];
            const float2 cc = s_c[j];
            float p2[P];
            bool ok[P];
            bool any = false;
            RowGroup rgp[NG];  // every aligned group of 4 rows has its own base, whatever P is
#pragma unroll
            for (int gq = 0; gq < NG; ++gq) rgp[gq] = row_group(a, bb, fx, fyg + 4.0f * (float)gq);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                p2[p] = row_p2(rgp[(q0 + p) >> 2], bb, (q0 + p) & 3);
                ok[p] = !done[p] && p2[p] <= 0.0f && p2[p] >= cc.y;
                any = any || ok[p];
            }
            if (__any_sync(0xffffffffu, any)) {
                const unsigned idx = (unsigned)(b0 + j + 1);
                // the P pixels update independently (predicated, no branches) so they interleave
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const float alpha = fminf(kAlphaMax, bb.y * fast_ex2(p2[p]));
                    const bool okp = ok[p] && alpha >= kAlphaMin;
                    const float Tn = T[p] * (1.0f - alpha);
                    const bool stop = okp && Tn < kTMin;
                    const bool add = okp && !stop;
                    const float w = add ? alpha * T[p] : 0.0f;
                    C0[p] = fmaf(w, bb.z, C0[p]);
                    C1[p] = fmaf(w, bb.w, C1[p]);
                    C2[p] = fmaf(w, cc.x, C2[p]);
                    T[p] = add ? Tn : T[p];
                    last[p] = add ? idx : last[p];
                    done[p] = done[p] || stop;
                }
            }
            if ((j & 7) == 7) {
                bool mine = true;
#pragma unroll
                for (int p = 0; p < P; ++p) mine = mine && done[p];
                if (__all_sync(0xffffffffu, mine)) break;
            }
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p)
        if (inside[p]) {
            const int py = py0 + p;
            const long long pix = cam.pix0 + (long long)py * cam.W + px;
            rgba[pix] = make_float4(C0[p] + T[p] * bg.x, C1[p] + T[p] * bg.y, C2[p] + T[p] * bg.z, 1.0f - T[p]);
            final_T[pix] = T[p];
            last_out[pix] = last[p];
        }
}

cudaError_t launch_render(const ivrgs_projected* p, const ivrgs_bins* b, const CamBatch& cb, const float* bg,
                          float* rgba, float* final_T, uint32_t* last, cudaStream_t s) {
    if (cb.n_tiles == 0) return cudaSuccess;
    IVRGS_PROF("k_render", s);
    const float2* xy = reinterpret_cast<const float2*>(p->xy);
    const float4* co = reinterpret_cast<const float4*>(p->conic_o);
    const float4* cd = reinterpret_cast<const float4*>(p->rgbd);
    const uint2* rg = reinterpret_cast<const uint2*>(b->ranges);
    const float3 bgc = make_float3(bg[0], bg[1], bg[2]);
    float4* out = reinterpret_cast<float4*>(rgba);
    const int ppt = blend_ppt(options().render_ppt, cb.n_tiles, false);
    if (ppt == 1)
        k_render<1><<<(unsigned)cb.n_tiles, kTilePix, 0, s>>>(xy, co, cd, p->n, b->values, rg, cb, bgc, out, final_T,
                                                             last);
    else if (ppt == 8)
        k_render<8><<<(unsigned)cb.n_tiles, kTilePix / 8, 0, s>>>(xy, co, cd, p->n, b->values, rg, cb, bgc, out,
                                                                 final_T, last);
    else if (ppt == 4)
        k_render<4><<<(unsigned)cb.n_tiles, kTilePix / 4, 0, s>>>(xy, co, cd, p->n, b->values, rg, cb, bgc, out,
                                                                 final_T, last);
    else
        k_render<2><<<(unsigned)cb.n_tiles, kTilePix / 2, 0, s>>>(xy, co, cd, p->n, b->values, rg, cb, bgc, out,
                                                                 final_T, last);
    return cudaGetLastError();
}

}  // namespace ivrgs

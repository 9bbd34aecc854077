// Per-tile front-to-back compositing (row a5; Sec. 3 second equation).
//
// One CTA of 256 threads per 16x16 tile, one pixel per thread. The tile's sorted run is
// walked in batches of 256 Gaussians: each thread stages one Gaussian into shared memory
// (mean, conic pre-scaled by -log2(e)/2 so that the exponent is one FMA chain, opacity,
// colour), then every pixel walks the batch. The CTA leaves as soon as every pixel has
// reached T < 1e-4 (barrier count).
#include "blend_alpha.cuh"

namespace ivrgs {

__global__ void __launch_bounds__(kTilePix) k_render(const float2* __restrict__ xy, const float4* __restrict__ conic_o,
                                                     const float4* __restrict__ rgbd, long long n,
                                                     const unsigned* __restrict__ values,
                                                     const uint2* __restrict__ ranges,
                                                     const __grid_constant__ CamBatch cb, float3 bg,
                                                     float4* __restrict__ rgba, float* __restrict__ final_T,
                                                     unsigned* __restrict__ last_out) {
    __shared__ float4 s_a[kTilePix];
    __shared__ float4 s_b[kTilePix];
    __shared__ float s_blue[kTilePix];
    const long long tile = blockIdx.x;
    const int v = view_of_tile(cb, tile);
    const CamDev& cam = cb.c[v];
    const int local = (int)(tile - cam.tile0);
    const int tx = local % cam.gx, ty = local / cam.gx;
    const int px = tx * kTile + (threadIdx.x & (kTile - 1));
    const int py = ty * kTile + (threadIdx.x / kTile);
    const bool inside = px < cam.W && py < cam.H;
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    const uint2 rg = ranges[tile];
    const long long vbase = (long long)v * n;

    float C0 = 0.f, C1 = 0.f, C2 = 0.f, T = 1.f;
    unsigned last = 0;
    bool done = !inside;
    const int len = (int)(rg.y - rg.x);
    for (int b0 = 0; b0 < len; b0 += kTilePix) {
        if (__syncthreads_count(done) == kTilePix) break;
        const int e = b0 + (int)threadIdx.x;
        if (e < len) {
            const unsigned g = values[rg.x + e];
            float4 sa, sb;
            float4 cd = make_float4(0.f, 0.f, 0.f, 0.f);
            if (g < (unsigned long long)n) {
                const long long gi = vbase + g;
                cd = rgbd[gi];
                stage_gaussian(xy[gi], conic_o[gi], cd, sa, sb);
            } else {  // never for a completed sort; a zero-opacity stand-in keeps reads in bounds
                stage_gaussian(make_float2(0.f, 0.f), make_float4(1.f, 0.f, 1.f, 0.f), cd, sa, sb);
            }
            s_a[threadIdx.x] = sa;
            s_b[threadIdx.x] = sb;
            s_blue[threadIdx.x] = cd.z;
        }
        __syncthreads();
        const int cnt = min(kTilePix, len - b0);
        if (!done) {
            for (int j = 0; j < cnt; ++j) {
                const float4 a = s_a[j];
                const float4 bb = s_b[j];
                float dx, dy;
                const float p2 = blend_p2(a, bb, fx, fy, dx, dy);
                if (p2 > 0.0f) continue;
                const float alpha = fminf(kAlphaMax, bb.y * fast_ex2(p2));
                if (alpha < kAlphaMin) continue;
                const float Tn = T * (1.0f - alpha);
                if (Tn < kTMin) {
                    done = true;
                    break;
                }
                const float w = alpha * T;
                C0 = fmaf(w, bb.z, C0);
                C1 = fmaf(w, bb.w, C1);
                C2 = fmaf(w, s_blue[j], C2);
                T = Tn;
                last = (unsigned)(b0 + j + 1);
            }
        }
    }
    if (inside) {
        const long long pix = cam.pix0 + (long long)py * cam.W + px;
        rgba[pix] = make_float4(C0 + T * bg.x, C1 + T * bg.y, C2 + T * bg.z, 1.0f - T);
        final_T[pix] = T;
        last_out[pix] = last;
    }
}

cudaError_t launch_render(const ivrgs_projected* p, const ivrgs_bins* b, const CamBatch& cb, const float* bg,
                          float* rgba, float* final_T, uint32_t* last, cudaStream_t s) {
    if (cb.n_tiles == 0) return cudaSuccess;
    {
        IVRGS_PROF("k_render", s);
        k_render<<<(unsigned)cb.n_tiles, kTilePix, 0, s>>>(
            reinterpret_cast<const float2*>(p->xy), reinterpret_cast<const float4*>(p->conic_o),
            reinterpret_cast<const float4*>(p->rgbd), p->n, b->values, reinterpret_cast<const uint2*>(b->ranges), cb,
            make_float3(bg[0], bg[1], bg[2]), reinterpret_cast<float4*>(rgba), final_T, last);
    }
    return cudaGetLastError();
}

}  // namespace ivrgs

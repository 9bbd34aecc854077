// The per-(pixel, Gaussian) alpha of the compositing, shared by the forward and the backward
// blend so that both take identical float32 decisions (skip, cut-off, termination).
#pragma once

#include "common.cuh"

namespace ivrgs {

// staged Gaussian: sa = (u, v, A', B'), sb = (C', o', r, g), sc = (b, p2_skip) with
// A' = -a log2e / 2, B' = -b log2e, C' = -c log2e / 2 (so that p2 = log2(e) * P is one FMA
// chain) and p2_skip = log2(1 / (255 o')) - 1e-3: below it o' 2^p2 < 1/255 for certain (the
// margin covers the rounding of log2 and of ex2.approx by orders of magnitude), so the entry
// can be skipped before the exponential without changing any decision.
__device__ __forceinline__ void stage_gaussian(const float2 m, const float4 co, const float4 cd, float4& sa,
                                               float4& sb, float2& sc) {
    sa = make_float4(m.x, m.y, (-0.5f * kLog2e) * co.x, (-kLog2e) * co.y);
    sb = make_float4((-0.5f * kLog2e) * co.z, co.w, cd.x, cd.y);
    const float thr = co.w > 0.0f ? -log2f(255.0f * co.w) - 1e-3f : -INFINITY;
    sc = make_float2(cd.z, co.w > 0.0f ? thr : INFINITY);
}

// returns p2 = log2(e) * P and writes dx = u - px, dy = v - py
__device__ __forceinline__ float blend_p2(const float4& sa, const float4& sb, float fx, float fy, float& dx,
                                          float& dy) {
    dx = sa.x - fx;
    dy = sa.y - fy;
    return fmaf(sa.z * dx, dx, fmaf(sa.w * dx, dy, sb.x * dy * dy));
}

}  // namespace ivrgs

// The per-(pixel, Gaussian) alpha of the compositing, shared by the forward and the backward
// blend so that both take identical float32 decisions (skip, cut-off, termination).
#pragma once

#include "common.cuh"

namespace ivrgs {

// staged Gaussian: sa = (u, v, A', B'), sb = (C', o', r, g) with A' = -a log2e / 2,
// B' = -b log2e, C' = -c log2e / 2 (so that p2 = log2(e) * P is one FMA chain)
__device__ __forceinline__ void stage_gaussian(const float2 m, const float4 co, const float4 cd, float4& sa,
                                               float4& sb) {
    sa = make_float4(m.x, m.y, (-0.5f * kLog2e) * co.x, (-kLog2e) * co.y);
    sb = make_float4((-0.5f * kLog2e) * co.z, co.w, cd.x, cd.y);
}

// returns p2 = log2(e) * P and writes dx = u - px, dy = v - py
__device__ __forceinline__ float blend_p2(const float4& sa, const float4& sb, float fx, float fy, float& dx,
                                          float& dy) {
    dx = sa.x - fx;
    dy = sa.y - fy;
    return fmaf(sa.z * dx, dx, fmaf(sa.w * dx, dy, sb.x * dy * dy));
}

}  // namespace ivrgs

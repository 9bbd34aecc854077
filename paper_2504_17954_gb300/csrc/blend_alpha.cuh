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

// p2 = log2(e) * P over an aligned group of 4 pixel rows of one column. With dx = u - px and
// dy0 = v - py0 at the group's first row, row py0 + p has dy = dy0 - p and
//   p2(p) = base - p k1 + p^2 C',  base = A' dx^2 + B' dx dy0 + C' dy0^2,  k1 = B' dx + 2 C' dy0.
// Forward and backward evaluate exactly these fused operations for every pixel, whatever the
// number of pixels per thread, so their float32 decisions agree bit for bit.
struct RowGroup {
    float dx, dy0, base, k1;
};

__device__ __forceinline__ RowGroup row_group(const float4& sa, const float4& sb, float fx, float fy0) {
    RowGroup q;
    q.dx = sa.x - fx;
    q.dy0 = sa.y - fy0;
    q.base = fmaf(sa.z * q.dx, q.dx, fmaf(sa.w * q.dx, q.dy0, sb.x * q.dy0 * q.dy0));
    q.k1 = fmaf(2.0f * sb.x, q.dy0, sa.w * q.dx);
    return q;
}

__device__ __forceinline__ float row_p2(const RowGroup& q, const float4& sb, int p) {
    return fmaf(sb.x, (float)(p * p), fmaf(-(float)p, q.k1, q.base));
}

__device__ __forceinline__ float fast_rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

}  // namespace ivrgs

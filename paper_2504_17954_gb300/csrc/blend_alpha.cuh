// The per-(pixel, Gaussian) alpha of the compositing, shared by the forward and the backward
// blend so that both take identical float32 decisions (skip, cut-off, termination).
#pragma once

#include <type_traits>

#include "common.cuh"

namespace ivrgs {

// The exponent P = -(a dx^2 + 2 b dx dy + c dy^2) / 2 of the conic K = (a, b; b, c) is evaluated
// in its completed-square form P = -(c y^2 + g dx^2) / 2 with y = dy + (b / c) dx and
// g = a - b^2 / c (the record holds (g, b, c, o')): two non-negative terms, so for long, thin
// Gaussians the small values of P along the long axis are not differences of large terms (in
// float32 the expanded form loses ~1e-3 of P at an axis ratio of 80, this one ~3e-5).
//
// staged Gaussian: sa = (u, v, C', beta), sb = (G', o', r, g), sc = (b, mid) with
// C' = -c log2e / 2, beta = b / c, G' = -g log2e / 2 (so that p2 = log2(e) * P = C' y^2 + G' dx^2)
// and mid = thr / 2, thr = log2(1 / (255 o')). The compositing's two range rules are decided on
// the exponent, before the exponential: the P > 0 guard (p2 <= 0) and the 1/255 cut-off, since
// o' 2^p2 >= 1/255 exactly when p2 >= thr. In float32 this decides the cut-off otherwise than
// the exact alpha only within a few ulp of thr (the rounding of log2f, of p2 and of ex2.approx),
// a float64 near-tie of |ln(255 alpha)| far below 1e-3. The range test is one compare,
// |p2 - mid| <= -mid (in_reach); mid is NaN for o' <= 0, so that nothing is in reach.
__device__ __forceinline__ void stage_gaussian(const float2 m, const float4 co, const float4 cd, float4& sa,
                                               float4& sb, float2& sc) {
    sa = make_float4(m.x, m.y, (-0.5f * kLog2e) * co.z, co.y / co.z);
    sb = make_float4((-0.5f * kLog2e) * co.x, co.w, cd.x, cd.y);
    const float thr = co.w > 0.0f ? -log2f(255.0f * co.w) : 0.0f;
    sc = make_float2(cd.z, co.w > 0.0f ? 0.5f * thr : __int_as_float(0x7fc00000));
}

// Rows a staged Gaussian can reach: the cut-off ellipse p2 >= thr is, in (dx, y) with
// y = dy + beta dx, the axis-aligned |C'| y^2 + |G'| dx^2 <= |thr|, whose extent in dy is
// +-H, H = sqrt(|thr| (1 / |C'| + beta^2 / |G'|)) (the support of that ellipse in the direction
// (-beta, 1)). Returned as (v - H', v + H') with H' = H (1 + 2^-8) + 2^-6 px, a margin far above
// the float32 rounding of H and of p2, so that no pixel row outside it can pass in_reach. NaN
// (no row) when nothing is in reach (o' <= 1/255 or o' <= 0); +-inf for a degenerate conic.
__device__ __forceinline__ float2 reach_rows(const float4& sa, const float4& sb, const float2& sc) {
    const float t = -2.0f * sc.y;  // |thr|
    const float h2 = t * (1.0f / (-sa.z) + sa.w * sa.w / (-sb.x));
    const float H = fmaf(sqrtf(h2), 1.0f + 0.00390625f, 0.015625f);
    return make_float2(sa.y - H, sa.y + H);
}

// Whether a blend walking P pixels per thread compacts each batch to the entries that reach its
// warp's rows first: with 1 or 2 pixels per thread a warp covers 2 or 4 of the tile's 16 rows
// and skips most entries of a long run that way (measured on the single 800^2 view: forward
// 0.475 -> 0.447 ms, backward 0.699 -> 0.647 ms); with 4 a warp covers half the tile, and the
// list's registers cost the backward more than the skipped entries save (1.47 -> 1.53 ms on the
// 8-view workload).
template <int P>
constexpr bool band_cull() { return P <= 2; }

// The slots [j0, j1) of a staged batch whose reach rows meet the pixel-centre rows [ylo, yhi]
// of this warp, in slot order, written to list (one warp's array of at least j1 - j0 bytes);
// returns their number (the same in every lane).
__device__ __forceinline__ int band_list(int j0, int j1, float ylo, float yhi, const float2* s_rows,
                                         unsigned char* list) {
    const int lane = threadIdx.x & 31;
    int n = 0;
    for (int q = j0; q < j1; q += 32) {
        const int j = q + lane;
        bool hit = false;
        if (j < j1) {
            const float2 r = s_rows[j];
            hit = r.x <= yhi && r.y >= ylo;
        }
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (hit) list[n + __popc(m & ((1u << lane) - 1u))] = (unsigned char)j;
        n += __popc(m);
    }
    __syncwarp();
    return n;
}

// Opacities o' at or below this never reach the 0.99 alpha clamp: in_reach admits p2 <= 0 up to
// the rounding of p2 - mid (below 1e-6), and ex2.approx errs by under 2^-22, so o' 2^p2 stays
// below 0.99. A staged entry is the same for the whole warp, so the blends branch on it
// uniformly and drop the clamp (and, backward, its zero derivative) for such Gaussians (1M
// Gaussians / 8 views: forward 0.783 -> 0.730 ms; backward 1.228 -> 1.209 ms together with its
// weight taken as the rise of T).
constexpr float kNoClampOpacity = kAlphaMax * (1.0f - 1.0f / 524288.0f);

// 1 - alpha of an entry of opacity o' with G = 2^p2, alpha = min(0.99, o' G), in explicitly
// rounded operations so that every walk that keeps T (the forward blend, the auxiliary maps)
// gets the same bits: with the clamp, 1 - fl(min(0.99, o' G)); without it (o' <=
// kNoClampOpacity), fl(1 - o' G) in one fused operation.
template <bool CLAMP>
__device__ __forceinline__ float one_minus_alpha(float o, float G) {
    return CLAMP ? __fsub_rn(1.0f, fminf(kAlphaMax, __fmul_rn(o, G))) : __fmaf_rn(-o, G, 1.0f);
}

// p2 in [2 mid, 0]: the entry is composited (up to the rounding of p2 - mid, which moves the
// ends by an ulp of mid: a float32 near-tie of the cut-off, or P ~ 0 at the centre, one of the
// P > 0 guard)
__device__ __forceinline__ bool in_reach(float p2, float mid) { return fabsf(__fsub_rn(p2, mid)) <= -mid; }

// p2 = log2(e) * P over an aligned group of 4 pixel rows of one column. With dx = u - px and
// dy0 = v - py0 at the group's first row, row py0 + p has dy = dy0 - p, y = y0 - p with
// y0 = dy0 + beta dx, and
//   p2(p) = C' (y0 - p)^2 + G' dx^2 = base - p k1 + p^2 C',  base = C' y0^2 + G' dx^2,  k1 = 2 C' y0.
// base is a sum of two non-negative terms, and with p <= 3 the expansion over the group's rows
// adds only rounding of the order of C' itself. Forward and backward evaluate exactly these
// explicitly rounded operations (no contraction or reordering can make them differ) for every
// pixel, whatever the number of pixels per thread, so their float32 decisions agree bit for bit.
struct RowGroup {
    float dx, dy0, base, k1;
};

__device__ __forceinline__ RowGroup row_group(const float4& sa, const float4& sb, float fx, float fy0) {
    RowGroup q;
    q.dx = __fsub_rn(sa.x, fx);
    q.dy0 = __fsub_rn(sa.y, fy0);
    const float y0 = __fmaf_rn(sa.w, q.dx, q.dy0);
    const float cy = __fmul_rn(sa.z, y0);
    q.base = __fmaf_rn(cy, y0, __fmul_rn(__fmul_rn(sb.x, q.dx), q.dx));
    q.k1 = __fmul_rn(2.0f, cy);
    return q;
}

__device__ __forceinline__ float row_p2(const RowGroup& q, const float4& sa, int p) {
    if (p == 0) return q.base;  // the expansion's terms are +-0 there (C' and k1 finite)
    return __fmaf_rn(sa.z, (float)(p * p), __fmaf_rn(-(float)p, q.k1, q.base));
}

// Calls f(P, TH) with the launch shape as integral constants: P pixels per thread (1, 2, 4 or 8),
// tiles TH = 16 or 8 pixels high; with 8-pixel-high tiles at most 4 pixels per thread, so that a
// tile keeps a full warp for the walks' votes (8 is taken as 4).
template <typename F>
inline void blend_shape(int ppt, int th, F&& f) {
    using std::integral_constant;
    if (th == 8) {
        if (ppt == 1) f(integral_constant<int, 1>{}, integral_constant<int, 8>{});
        else if (ppt == 2) f(integral_constant<int, 2>{}, integral_constant<int, 8>{});
        else f(integral_constant<int, 4>{}, integral_constant<int, 8>{});
        return;
    }
    if (ppt == 1) f(integral_constant<int, 1>{}, integral_constant<int, 16>{});
    else if (ppt == 2) f(integral_constant<int, 2>{}, integral_constant<int, 16>{});
    else if (ppt == 8) f(integral_constant<int, 8>{}, integral_constant<int, 16>{});
    else f(integral_constant<int, 4>{}, integral_constant<int, 16>{});
}

// Position of a thread's pixels in its tile.
struct TilePos {
    int px, py0, q0;
    float fx, fyg;
};

template <int P, int TH>
__device__ __forceinline__ TilePos tile_pos(const CamDev& cam, long long tile) {
    TilePos t;
    const int local = (int)(tile - cam.tile0);
    const int tx = local % cam.gx, ty = local / cam.gx;
    t.px = tx * kTile + (threadIdx.x & (kTile - 1));
    t.py0 = ty * TH + (threadIdx.x / kTile) * P;
    t.fx = (float)t.px + 0.5f;
    t.q0 = t.py0 & 3;                              // offset of this thread's first row in its group
    t.fyg = (float)(t.py0 - t.q0) + 0.5f;          // centre of the group's first row
    return t;
}

// Split walk of a long run over a cluster of kSplit CTAs: a run of len entries is cut into nc
// chunks of equal length (nc = 1 up to split_min entries, else ceil(len / split_min), at most
// kSplit); CTA `rank` takes [lo, hi).
constexpr int kSplit = 8;

__device__ __forceinline__ void split_chunk(int len, int split_min, int rank, int& nc, int& lo, int& hi) {
    nc = len <= split_min ? 1 : min(kSplit, (len + split_min - 1) / split_min);
    const int ch = (len + nc - 1) / nc;
    lo = min(len, rank * ch);
    hi = min(len, lo + ch);
}

__device__ __forceinline__ float fast_rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

}  // namespace ivrgs

// Tile culling by the opacity cut-off ellipse (IVRGS_BIN_CULL).
//
// The compositing skips a Gaussian wherever alpha = min(0.99, o' G) < 1/255 (Sec. 3 blend, with
// the 1/255 threshold of 3DGS). With conic (a, b, c) (the record holds (g, b, c, o'), g = a -
// b^2 / c, so a = g + b^2 / c and det = a c - b^2 = g c without cancellation), e = pixel - centre and
// q(e) = a e_x^2 + 2 b e_x e_y + c e_y^2 we have G = exp(-q/2), so the Gaussian changes no pixel
// where q > tau = 2 ln(255 o'). A tile of its square rectangle in which every pixel centre has
// q > tau can therefore be dropped from the tile lists without changing any composited value,
// transmittance or gradient: it would be skipped at every pixel of that tile.
//
// Per tile row the kept tiles are the columns whose box of pixel centres
// [16 tx + 0.5, 16 tx + 15.5] meets the ellipse q <= tau' (tau' = tau + kCullSlack) within the
// row's band of pixel-centre rows [th ty + 0.5, th ty + th - 0.5] (th the tile height). For one e_y the ellipse's chord
// is centred at -(b/a) e_y with half width sqrt(tau' a - det e_y^2) / a (det = a c - b^2). Over
// a band of e_y its leftmost end lies at the e_y of the ellipse's leftmost point,
// e_y = (b/c) X with X = sqrt(tau' c / det), clamped into the band (the left end is a convex
// function of e_y), and its rightmost end at the clamped e_y = -(b/c) X (the right end is
// concave). Every step is an explicitly rounded float32 operation or a hardware approximation
// (reciprocal, reciprocal square root, log2), each a fixed function of its input, so the
// counting and emission kernels reach identical decisions; the approximations' relative errors
// (below 1e-6) are far inside the slack.
//
// Conservativeness: kCullSlack raises the cut-off by a factor e^(kCullSlack / 2) in alpha, and
// every pixel centre of a tile lies in its box. For a conic with a c <= kCullCond det, float32
// rounding in q (here and in the blend) stays far below the slack; more elongated conics,
// non-finite inputs and non-positive conics keep their whole rectangle.
#pragma once

#include "common.cuh"

namespace ivrgs {

constexpr float kCullSlack = 0.25f;
constexpr float kCullCond = 4096.0f;

__device__ __forceinline__ float cull_sqrt(float x) { return x > 0.0f ? __fmul_rn(x, rsqrtf(x)) : 0.0f; }
__device__ __forceinline__ float cull_div(float a, float b) { return __fdividef(a, b); }

struct CullEll {
    float u, v;    // centre (pixels)
    float ba;      // b / a
    float inv_a;   // 1 / a
    float ta;      // tau' a
    float det;     // a c - b^2
    float Y;       // half height of the ellipse q <= tau'
    float eyR;     // e_y of its rightmost point (the leftmost point is at -eyR)
    int mode;      // 0: no pixel reaches 1/255; 1: cull by rows; 2: keep the whole rectangle
};

__device__ __forceinline__ CullEll cull_setup(float2 uv, float4 co, int enabled) {
    CullEll e;
    e.u = uv.x;
    e.v = uv.y;
    e.ba = e.inv_a = e.ta = e.det = e.Y = e.eyR = 0.0f;
    e.mode = 2;
    if (!enabled) return e;
    const float g = co.x, b = co.y, c = co.z, o = co.w;
    if (!(isfinite(g) && isfinite(b) && isfinite(c) && isfinite(o) && isfinite(uv.x) && isfinite(uv.y))) return e;
    const float s = __fmul_rn(255.0f, o);
    if (!(s > 0.0f)) {  // o' <= 0: alpha = 0 everywhere
        e.mode = 0;
        return e;
    }
    const float tau = __fadd_rn(__fmul_rn(2.0f, __logf(s)), kCullSlack);
    if (!(tau > 0.0f)) {  // o' < e^(-kCullSlack / 2) / 255: alpha < 1/255 everywhere
        e.mode = 0;
        return e;
    }
    if (!(c > 0.0f)) return e;
    const float a = __fmaf_rn(b, __fdiv_rn(b, c), g);
    const float det = __fmul_rn(g, c);
    if (!(a > 0.0f) || !(det > 0.0f) || !isfinite(a) || __fmul_rn(a, c) > __fmul_rn(kCullCond, det)) return e;
    e.inv_a = cull_div(1.0f, a);
    e.ba = __fmul_rn(b, e.inv_a);
    e.ta = __fmul_rn(tau, a);
    e.det = det;
    const float inv_det = cull_div(1.0f, det);
    e.Y = cull_sqrt(__fmul_rn(e.ta, inv_det));
    const float X = cull_sqrt(__fmul_rn(__fmul_rn(tau, c), inv_det));
    e.eyR = -__fmul_rn(cull_div(b, c), X);
    e.mode = 1;
    return e;
}

// pixel x of the chord end at e_y: centre - (b/a) e_y +- half width
__device__ __forceinline__ float cull_chord_end(const CullEll& e, float ey, float sign) {
    const float w2 = __fsub_rn(e.ta, __fmul_rn(e.det, __fmul_rn(ey, ey)));
    const float hw = __fmul_rn(cull_sqrt(w2), e.inv_a);
    return __fadd_rn(__fsub_rn(e.u, __fmul_rn(e.ba, ey)), __fmul_rn(sign, hw));
}

// kept tile columns [lo, hi) of tile row ty (tiles th pixels high) within the rectangle's columns [x0, x1)
__device__ __forceinline__ void cull_row(const CullEll& e, int ty, int th, int x0, int x1, int& lo, int& hi) {
    if (e.mode == 2) {
        lo = x0;
        hi = x1;
        return;
    }
    lo = hi = x0;
    if (e.mode == 0) return;
    const float band0 = __fsub_rn(__fadd_rn((float)(ty * th), 0.5f), e.v);
    const float y0 = fmaxf(band0, -e.Y);
    const float y1 = fminf(__fadd_rn(band0, (float)(th - 1)), e.Y);
    if (!(y0 <= y1)) return;
    const float eyR = fminf(fmaxf(e.eyR, y0), y1);
    const float eyL = fminf(fmaxf(-e.eyR, y0), y1);
    const float xl = cull_chord_end(e, eyL, -1.0f);
    const float xr = cull_chord_end(e, eyR, 1.0f);
    // columns tx with 16 tx + 0.5 <= xr and 16 tx + 15.5 >= xl
    const float inv = 1.0f / (float)kTile;  // exact: power of two
    const float fl = fminf(fmaxf(ceilf(__fmul_rn(__fsub_rn(xl, (float)kTile - 0.5f), inv)), (float)x0), (float)x1);
    const float fh = fminf(fmaxf(floorf(__fmul_rn(__fsub_rn(xr, 0.5f), inv)) + 1.0f, (float)x0), (float)x1);
    lo = (int)fl;
    hi = (int)fh;
    if (hi < lo) hi = lo;
}

}  // namespace ivrgs

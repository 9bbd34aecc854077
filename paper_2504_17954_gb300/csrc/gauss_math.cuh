// Per-Gaussian projection and shading math (float32, one thread per Gaussian), shared by
// the forward projection kernel and the backward kernel, which recomputes it.
//   Sec. 3: Sigma = R(q) S S^T R(q)^T, Sigma' = J W Sigma W^T J^T (+ lowpass I), 2D mean
//   through the pinhole; Blinn-Phong c = k_a c_v + k_d c_v |n.l| + [|n.l|>0] k_s |n.h|^beta.
//   Sec. 4.3: c_v = c_p + dc.  Sec. 4.5/4.6: o' = s_m sigmoid(logit), k' = lambda k + b.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace ivrgs {

// view-independent quantities of one Gaussian
struct GaussLocal {
    float mu[3];
    float qn[4], qlen;       // normalised quaternion, |q|
    float Rq[9];            // rotation of qn
    float sc[3];            // exp(log s)
    float nn[3], nlen;      // normalised normal, |n|
    float cv[3];            // c_p + dc
    float k[4], kp[4];      // stored k and edited k' = lambda k + b
    float sig, o;           // sigmoid(logit), o' = s_m sigmoid
    float sm;               // opacity scale of the model
    float tl[3], tl_len;    // the edit table's global light, normalised, and its length
    bool tl_on;             // the global light replaces every orbital view's light_dir
    const float* sh;        // this Gaussian's SH coefficients [nb][3] (3DGS colour) or nullptr
    int sh_deg;
    int model;
    bool visible;
};

// codebook value of attribute a (0 log_scale, 1 quat, 2 opacity_logit, 3 dcolor, 4..7 k_a..beta)
// of model m for the uint8 index q (IVRGS_VQ storage)
__device__ __forceinline__ float vq_value(const ivrgs_gaussians& g, int m, int a, unsigned q) {
    return __ldg(g.codebook + ((long long)m * IVRGS_VQ_ATTRS + a) * g.vq_k + q);
}

// attribute loads: float32 storage, the 16-bit IVRGS_MIXED storage or the IVRGS_VQ codebook
// indices, decoded to float32 (m = model of Gaussian i, used by IVRGS_VQ)
template <int PREC>
__device__ __forceinline__ void load_attrs(const ivrgs_gaussians& g, long long i, int m, float mu[3], float4& q,
                                           float ls[3], float& logit, float dc[3], float nrm[3], float4& kk) {
    if constexpr (PREC == IVRGS_VQ) {
        const float* mf = static_cast<const float*>(g.mean);
        const float* nf = static_cast<const float*>(g.normal);
        const unsigned char* si = static_cast<const unsigned char*>(g.log_scale);
        const unsigned char* ci = static_cast<const unsigned char*>(g.dcolor);
        const uchar4 qi = static_cast<const uchar4*>(g.quat)[i];
        const uchar4 ki = static_cast<const uchar4*>(g.kads)[i];
        for (int k = 0; k < 3; ++k) {
            mu[k] = mf[3 * i + k];
            nrm[k] = nf[3 * i + k];
            ls[k] = vq_value(g, m, 0, si[3 * i + k]);
            dc[k] = vq_value(g, m, 3, ci[3 * i + k]);
        }
        q = make_float4(vq_value(g, m, 1, qi.x), vq_value(g, m, 1, qi.y), vq_value(g, m, 1, qi.z),
                        vq_value(g, m, 1, qi.w));
        logit = vq_value(g, m, 2, static_cast<const unsigned char*>(g.opacity_logit)[i]);
        kk = make_float4(vq_value(g, m, 4, ki.x), vq_value(g, m, 5, ki.y), vq_value(g, m, 6, ki.z),
                         vq_value(g, m, 7, ki.w));
    } else if constexpr (PREC == IVRGS_FP32) {
        const float* m = static_cast<const float*>(g.mean);
        const float* s = static_cast<const float*>(g.log_scale);
        const float* c = static_cast<const float*>(g.dcolor);
        const float* n = static_cast<const float*>(g.normal);
        for (int k = 0; k < 3; ++k) {
            mu[k] = m[3 * i + k];
            ls[k] = s[3 * i + k];
            dc[k] = c[3 * i + k];
            nrm[k] = n[3 * i + k];
        }
        q = static_cast<const float4*>(g.quat)[i];
        kk = static_cast<const float4*>(g.kads)[i];
        logit = static_cast<const float*>(g.opacity_logit)[i];
    } else {
        const __half* m = static_cast<const __half*>(g.mean);
        const float* an = g.anchor + 3 * (i / IVRGS_ANCHOR_CHUNK);
        const __nv_bfloat16* s = static_cast<const __nv_bfloat16*>(g.log_scale);
        const __nv_bfloat16* c = static_cast<const __nv_bfloat16*>(g.dcolor);
        const __nv_bfloat16* n = static_cast<const __nv_bfloat16*>(g.normal);
        for (int k = 0; k < 3; ++k) {
            mu[k] = __fadd_rn(__ldg(an + k), __half2float(m[3 * i + k]));  // the stored mean: anchor + offset
            ls[k] = __bfloat162float(s[3 * i + k]);
            dc[k] = __bfloat162float(c[3 * i + k]);
            nrm[k] = __bfloat162float(n[3 * i + k]);
        }
        const uint2 qb = static_cast<const uint2*>(g.quat)[i];
        const __half2 q01 = *reinterpret_cast<const __half2*>(&qb.x), q23 = *reinterpret_cast<const __half2*>(&qb.y);
        q = make_float4(__low2float(q01), __high2float(q01), __low2float(q23), __high2float(q23));
        const uint2 kb = static_cast<const uint2*>(g.kads)[i];
        const __half2 k01 = *reinterpret_cast<const __half2*>(&kb.x), k23 = *reinterpret_cast<const __half2*>(&kb.y);
        kk = make_float4(__low2float(k01), __high2float(k01), __low2float(k23), __high2float(k23));
        logit = __half2float(static_cast<const __half*>(g.opacity_logit)[i]);
    }
}

template <int PREC>
__device__ __forceinline__ void load_gauss(const ivrgs_gaussians& g, const float* __restrict__ table, int n_models,
                                           long long i, GaussLocal& G) {
    G.model = g.model_id[i];
    const float* me = table + (long long)G.model * IVRGS_EDIT_STRIDE;
    G.visible = __ldg(me + 4) != 0.0f;
    float ls[3], dcol[3], nrm[3], logit;
    float4 q, kk;
    load_attrs<PREC>(g, i, G.model, G.mu, q, ls, logit, dcol, nrm, kk);
    G.qlen = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    const float iq = 1.0f / G.qlen;
    const float w = q.x * iq, x = q.y * iq, y = q.z * iq, z = q.w * iq;
    G.qn[0] = w; G.qn[1] = x; G.qn[2] = y; G.qn[3] = z;
    G.Rq[0] = 1.f - 2.f * (y * y + z * z); G.Rq[1] = 2.f * (x * y - w * z); G.Rq[2] = 2.f * (x * z + w * y);
    G.Rq[3] = 2.f * (x * y + w * z); G.Rq[4] = 1.f - 2.f * (x * x + z * z); G.Rq[5] = 2.f * (y * z - w * x);
    G.Rq[6] = 2.f * (x * z - w * y); G.Rq[7] = 2.f * (y * z + w * x); G.Rq[8] = 1.f - 2.f * (x * x + y * y);
    for (int k = 0; k < 3; ++k) G.sc[k] = expf(ls[k]);
    G.nlen = sqrtf(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
    const float inl = 1.0f / G.nlen;
    G.nn[0] = nrm[0] * inl; G.nn[1] = nrm[1] * inl; G.nn[2] = nrm[2] * inl;
    for (int c = 0; c < 3; ++c) G.cv[c] = __ldg(me + c) + dcol[c];
    G.k[0] = kk.x; G.k[1] = kk.y; G.k[2] = kk.z; G.k[3] = kk.w;
    const float* lam = table + (long long)n_models * IVRGS_EDIT_STRIDE;
    for (int c = 0; c < 4; ++c) G.kp[c] = __ldg(lam + c) * G.k[c] + __ldg(lam + 4 + c);
    G.sh = g.sh ? g.sh + i * 3ll * (g.sh_degree + 1) * (g.sh_degree + 1) : nullptr;
    G.sh_deg = g.sh_degree;
    G.tl_on = __ldg(lam + 11) != 0.0f;
    if (G.tl_on) {
        const float l0 = __ldg(lam + 8), l1 = __ldg(lam + 9), l2 = __ldg(lam + 10);
        G.tl_len = sqrtf(l0 * l0 + l1 * l1 + l2 * l2);
        const float il = 1.0f / G.tl_len;
        G.tl[0] = l0 * il; G.tl[1] = l1 * il; G.tl[2] = l2 * il;
    } else {
        G.tl[0] = G.tl[1] = G.tl[2] = 0.0f;
        G.tl_len = 1.0f;
    }
    G.sig = 1.0f / (1.0f + expf(-logit));
    G.sm = __ldg(me + 3);
    G.o = G.sm * G.sig;
}

// per-view quantities
struct ViewLocal {
    bool visible;
    float x, y, z, iz;
    float txc, tyc;
    bool clx, cly;
    float T[6];           // J W (2x3)
    float A, B, C, det;   // Sigma' (dilated) and its determinant
    float conic[3];       // K = Sigma'^-1 = (a, b; b, c)
    float gam;            // a - b^2 / c = 1 / A: K's completed-square form (the record's first entry)
    int radius;
    float u, v;
    float depth;
    // shading
    float vd[3], vlen, l[3], h[3], hlen;
    float ndl, ndh, nl, nh, spow;
    bool gate;
    float rgb[3];
    bool shc[3];  // SH colour clamped at 0 (per channel)
};

// Term t of the real SH basis below and its gradient, for unrolled loops (no arrays)
__device__ __forceinline__ float sh_term(int t, float x, float y, float z, float& gx, float& gy, float& gz) {
    const float PI = 3.14159265358979f;
    const float a = sqrtf(3.f / (4.f * PI)), b = sqrtf(15.f / (4.f * PI)), c = sqrtf(5.f / (16.f * PI)),
                e = sqrtf(15.f / (16.f * PI)), f = sqrtf(35.f / (32.f * PI)), g = sqrtf(105.f / (4.f * PI)),
                h = sqrtf(21.f / (32.f * PI)), k = sqrtf(7.f / (16.f * PI)), m = sqrtf(105.f / (16.f * PI));
    gx = gy = gz = 0.f;
    switch (t) {
        case 0: return 0.5f / sqrtf(PI);
        case 1: gy = -a; return -a * y;
        case 2: gz = a; return a * z;
        case 3: gx = -a; return -a * x;
        case 4: gx = b * y; gy = b * x; return b * x * y;
        case 5: gy = -b * z; gz = -b * y; return -b * y * z;
        case 6: gx = -2.f * c * x; gy = -2.f * c * y; gz = 4.f * c * z; return c * (2.f * z * z - x * x - y * y);
        case 7: gx = -b * z; gz = -b * x; return -b * x * z;
        case 8: gx = 2.f * e * x; gy = -2.f * e * y; return e * (x * x - y * y);
        case 9: gx = -6.f * f * x * y; gy = -f * (3.f * x * x - 3.f * y * y); return -f * y * (3.f * x * x - y * y);
        case 10: gx = g * y * z; gy = g * x * z; gz = g * x * y; return g * x * y * z;
        case 11:
            gx = 2.f * h * x * y; gy = -h * (4.f * z * z - x * x - 3.f * y * y); gz = -8.f * h * y * z;
            return -h * y * (4.f * z * z - x * x - y * y);
        case 12:
            gx = -6.f * k * x * z; gy = -6.f * k * y * z; gz = k * (6.f * z * z - 3.f * x * x - 3.f * y * y);
            return k * z * (2.f * z * z - 3.f * x * x - 3.f * y * y);
        case 13:
            gx = -h * (4.f * z * z - 3.f * x * x - y * y); gy = 2.f * h * x * y; gz = -8.f * h * x * z;
            return -h * x * (4.f * z * z - x * x - y * y);
        case 14: gx = 2.f * m * x * z; gy = -2.f * m * y * z; gz = m * (x * x - y * y); return m * z * (x * x - y * y);
        default: gx = -f * (3.f * x * x - 3.f * y * y); gy = 6.f * f * x * y; return -f * x * (x * x - 3.f * y * y);
    }
}

// sh_term: the real spherical harmonics up to degree 3 on a unit direction (x, y, z),
// orthonormal on the sphere, Condon-Shortley sign, normalisations written as their closed forms
// (sqrt(3/(4 pi)) etc.), term t and the gradient of its polynomial.

// Camera depth z = R20 mx + R21 my + R22 mz + t2 of float32 inputs, rounded once to float32.
// Compensated dot product (Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM J. Sci.
// Comput. 26(6), 2005, algorithm Dot2): every product is split exactly into p + e with one
// fused multiply-add, every running sum into s + e with Knuth's TwoSum, and the error terms are
// summed apart. s + c then lies within ~10 u^2 (|t2| + sum |R2k mk|) of the exact z (u = 2^-24),
// and the final addition, one correctly rounded float32 operation, returns the float32 nearest to
// z unless z lies that close to a midpoint between two floats. The sort key is thereby the exact
// depth rounded once, with no float64 arithmetic (which runs at a small fraction of the float32
// rate on this GPU). The _rn intrinsics keep the compiler from contracting or reordering.
__device__ __forceinline__ float camera_depth(const float R2[3], float t2, const float mu[3]) {
    float s = t2, c = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float p = __fmul_rn(R2[k], mu[k]);
        const float pe = __fmaf_rn(R2[k], mu[k], -p);  // R2k mk - p, exact
        const float s1 = __fadd_rn(s, p);
        const float bv = __fsub_rn(s1, s);
        const float se = __fadd_rn(__fsub_rn(s, __fsub_rn(s1, bv)), __fsub_rn(p, bv));  // s + p - s1, exact
        s = s1;
        c = __fadd_rn(c, __fadd_rn(se, pe));
    }
    return __fadd_rn(s, c);
}

// a d - b c with one rounding error (Kahan's algorithm for 2x2 determinants: the product b c is
// split exactly by an FMA, and its rounding error added back)
__device__ __forceinline__ float diff_of_products(float a, float d, float b, float c) {
    const float w = __fmul_rn(b, c);
    const float e = __fmaf_rn(-b, c, w);
    const float f = __fmaf_rn(a, d, -w);
    return __fadd_rn(f, e);
}

__device__ __forceinline__ void project_view(const GaussLocal& G, const CamDev& c, float lowpass, ViewLocal& V) {
    V.visible = false;
    // the sort key and the near-plane decision: the exact camera z rounded once to float32
    const float zd = camera_depth(c.R + 6, c.t[2], G.mu);
    if (!(zd > c.znear)) return;
    V.depth = zd;
    V.z = V.depth;
    V.x = fmaf(c.R[0], G.mu[0], fmaf(c.R[1], G.mu[1], fmaf(c.R[2], G.mu[2], c.t[0])));
    V.y = fmaf(c.R[3], G.mu[0], fmaf(c.R[4], G.mu[1], fmaf(c.R[5], G.mu[2], c.t[1])));
    V.iz = 1.0f / V.z;
    const float tx = V.x * V.iz, ty = V.y * V.iz;
    V.txc = fminf(fmaxf(tx, -c.limx), c.limx);
    V.tyc = fminf(fmaxf(ty, -c.limy), c.limy);
    V.clx = (tx < -c.limx) || (tx > c.limx);
    V.cly = (ty < -c.limy) || (ty > c.limy);
    const float J00 = c.fx * V.iz, J02 = -c.fx * V.txc * V.iz;
    const float J11 = c.fy * V.iz, J12 = -c.fy * V.tyc * V.iz;
    for (int j = 0; j < 3; ++j) {
        V.T[j] = J00 * c.R[j] + J02 * c.R[6 + j];
        V.T[3 + j] = J11 * c.R[3 + j] + J12 * c.R[6 + j];
    }
    // Sigma' = W W^T + lowpass I with W = T Rq diag(s) (2x3): A and C are sums of squares, B one
    // dot product, and det(W W^T) the sum of the squared 2x2 minors of W (Cauchy-Binet), so the
    // determinant is a sum of non-negative terms; for long, thin Gaussians the short axis of
    // Sigma' is then not lost to cancellation between A C and B^2
    float W0[3], W1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        W0[k] = (V.T[0] * G.Rq[k] + V.T[1] * G.Rq[3 + k] + V.T[2] * G.Rq[6 + k]) * G.sc[k];
        W1[k] = (V.T[3] * G.Rq[k] + V.T[4] * G.Rq[3 + k] + V.T[5] * G.Rq[6 + k]) * G.sc[k];
    }
    const float A0 = W0[0] * W0[0] + W0[1] * W0[1] + W0[2] * W0[2];
    const float C0 = W1[0] * W1[0] + W1[1] * W1[1] + W1[2] * W1[2];
    const float m01 = diff_of_products(W0[0], W1[1], W0[1], W1[0]);
    const float m02 = diff_of_products(W0[0], W1[2], W0[2], W1[0]);
    const float m12 = diff_of_products(W0[1], W1[2], W0[2], W1[1]);
    V.A = A0 + lowpass;
    V.B = W0[0] * W1[0] + W0[1] * W1[1] + W0[2] * W1[2];
    V.C = C0 + lowpass;
    V.det = fmaf(lowpass, A0 + C0 + lowpass, m01 * m01 + m02 * m02 + m12 * m12);
    if (!(V.det > 0.0f)) return;
    const float idet = 1.0f / V.det;
    V.conic[0] = V.C * idet;
    V.conic[1] = -V.B * idet;
    V.conic[2] = V.A * idet;
    V.gam = 1.0f / V.A;
    // lambda_max = (A + C)/2 + sqrt(((A - C)/2)^2 + B^2): the larger eigenvalue without cancellation
    const float mid = 0.5f * (V.A + V.C), hd = 0.5f * (V.A - V.C);
    const float lmax = mid + sqrtf(hd * hd + V.B * V.B);
    V.radius = (int)ceilf(3.0f * sqrtf(lmax));
    if (V.radius <= 0) return;
    V.u = c.fx * tx + c.cx;
    V.v = c.fy * ty + c.cy;
    // Blinn-Phong shading
    float d[3] = {c.campos[0] - G.mu[0], c.campos[1] - G.mu[1], c.campos[2] - G.mu[2]};
    V.vlen = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const float ivl = 1.0f / V.vlen;
    for (int k = 0; k < 3; ++k) V.vd[k] = d[k] * ivl;
    if (c.headlight) {
        for (int k = 0; k < 3; ++k) V.l[k] = V.vd[k];
    } else {
        for (int k = 0; k < 3; ++k) V.l[k] = G.tl_on ? G.tl[k] : c.light[k];
    }
    float hv[3] = {V.vd[0] + V.l[0], V.vd[1] + V.l[1], V.vd[2] + V.l[2]};
    V.hlen = sqrtf(hv[0] * hv[0] + hv[1] * hv[1] + hv[2] * hv[2]);
    const float ihl = V.hlen > 0.0f ? 1.0f / V.hlen : 0.0f;
    for (int k = 0; k < 3; ++k) V.h[k] = hv[k] * ihl;
    V.ndl = G.nn[0] * V.l[0] + G.nn[1] * V.l[1] + G.nn[2] * V.l[2];
    V.ndh = G.nn[0] * V.h[0] + G.nn[1] * V.h[1] + G.nn[2] * V.h[2];
    V.nl = fabsf(V.ndl);
    V.nh = fabsf(V.ndh);
    V.gate = (V.nl > 0.0f) && (V.nh > 0.0f);
    V.spow = V.gate ? __powf(V.nh, G.kp[3]) : 0.0f;  // nh in (0, 1]: exp2(beta log2 nh) on the MUFU
    const float spec = V.gate ? G.kp[2] * V.spow : 0.0f;
    const float diff = G.kp[0] + G.kp[1] * V.nl;
    for (int k = 0; k < 3; ++k) V.rgb[k] = diff * G.cv[k] + spec;
    if (G.sh) {  // 3DGS colour: SH of the direction from the camera (-vd), + 0.5, clamped at 0
        const int nb = (G.sh_deg + 1) * (G.sh_deg + 1);
        float v[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            if (t >= nb) break;
            float gx, gy, gz;
            const float Yt = sh_term(t, -V.vd[0], -V.vd[1], -V.vd[2], gx, gy, gz);
            for (int ch = 0; ch < 3; ++ch) v[ch] = fmaf(__ldg(G.sh + 3 * t + ch), Yt, v[ch]);
        }
        for (int ch = 0; ch < 3; ++ch) {
            V.shc[ch] = v[ch] < 0.0f;
            V.rgb[ch] = fmaxf(v[ch], 0.0f);
        }
    }
    V.visible = true;
}

}  // namespace ivrgs

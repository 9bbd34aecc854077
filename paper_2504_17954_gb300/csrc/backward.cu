// Reverse mode of the path (rows a6, a7).
//
// a6, per tile: every pixel walks its run back to front from its last contributor. The
// transmittance in front of contributor i is recovered from the stored final T as
// T_i = T_{i+1} / (1 - alpha_i) (not stored in the forward). With
// S_i = sum_{j>i} T_j alpha_j c_j + T_final bg, each contributor receives
//   dL/dc_i = T_i alpha_i dL/dC,
//   dL/dalpha_i = dL/dC . (T_i c_i - S_i / (1 - alpha_i)) + dL/dA T_final / (1 - alpha_i),
// chained through alpha = min(0.99, o' exp(P)) to (u, v), the conic and o'. The nine
// per-Gaussian sums are reduced across the warp (all lanes walk the same entry) and added
// with one vector atomic per warp.
//
// a7, per Gaussian: the projection and shading are recomputed per view; dL/dSigma (in the
// Gaussian's own frame), dL/dc_v, dL/dk', dL/dn and dL/do' are accumulated over views in
// registers and pushed through the view-independent parts (quaternion, scale, edits) once.
// The conic's gradient reaches Sigma' through the eigenbasis of Sigma', which keeps long, thin
// Gaussians' scale and rotation gradients free of cancellation in float32.
#include <climits>
#include <type_traits>
#include <cooperative_groups.h>

#include "blend_alpha.cuh"
#include "f32x2.cuh"
#include "gauss_math.cuh"

namespace cg = cooperative_groups;

namespace ivrgs {

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Sum of v[0..7] over the warp in 9 shuffles (recursive halving): on return every lane holds
// the warp total of value index (lane >> 2).
__device__ __forceinline__ float warp_sum8_transposed(const float v[8], int lane) {
    const bool b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1, b2 = (lane >> 2) & 1;
    float k1[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float send = b4 ? v[k] : v[4 + k];
        const float r = __shfl_xor_sync(0xffffffffu, send, 16);
        k1[k] = (b4 ? v[4 + k] : v[k]) + r;
    }
    float k2[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float send = b3 ? k1[k] : k1[2 + k];
        const float r = __shfl_xor_sync(0xffffffffu, send, 8);
        k2[k] = (b3 ? k1[2 + k] : k1[k]) + r;
    }
    float x;
    {
        const float send = b2 ? k2[0] : k2[1];
        const float r = __shfl_xor_sync(0xffffffffu, send, 4);
        x = (b2 ? k2[1] : k2[0]) + r;
    }
    x += __shfl_xor_sync(0xffffffffu, x, 2);
    x += __shfl_xor_sync(0xffffffffu, x, 1);
    return x;
}

// Per-thread state of the backward walk of P pixels: T just behind the entries still to walk
// (recovered by division while walking back), DS = dL/dC . S - dL/dA T_final with S the colour
// accumulated behind (sum over the contributors behind of T_j alpha_j c_j, plus T_final bg), the
// pixel's dL/dRGBA and its last contributor (1 + position in the run).
template <int P>
struct BwdPix {
    float T[P], DS[P];
    float4 d[P];
    unsigned my_last[P];
};

constexpr int kBwdBatch = 256;  // entries staged per batch

// Up to this many contributing lanes of a warp add their own record gradients to an entry's
// Gaussian (three vector atomics each) instead of reducing them across the warp first: fewer
// instructions than the nine-value transposed reduction, and the L2 takes the atomics. Beyond it
// the same-address atomics of a dense warp serialise at L2. Measured on GB300 (1M Gaussians /
// 8 views, backward blend): reduction from 2 lanes 1.40 ms; direct up to 8 / 16 / 24 / 28 lanes
// 1.32 / 1.27 / 1.23 / 1.25 ms; always direct 2.14 ms. The single 800^2 view: 1.43 -> 1.31 ms
// per step at 24.
constexpr int kDirectLanes = 24;
constexpr int kBwdSteps1 = 2;  // list entries per step of the one-pixel walk (1, 2 or 4)

// The backward state of this thread's P pixels from the forward's final T and last contributor
// and dL/dRGBA (DS = T_final (dL/dC . bg - dL/dA)); returns the largest last contributor.
template <int P>
__device__ __forceinline__ unsigned bwd_init(const CamDev& cam, int px, int py0, float3 bg,
                                             const float* __restrict__ final_T, const unsigned* __restrict__ last_in,
                                             const float4* __restrict__ dL, BwdPix<P>& st) {
    unsigned mx = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int py = py0 + p;
        float Tf = 1.0f;
        st.my_last[p] = 0;
        st.d[p] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (px < cam.W && py < cam.H) {
            const long long pix = cam.pix0 + (long long)py * cam.W + px;
            Tf = final_T[pix];
            st.my_last[p] = last_in[pix];
            st.d[p] = dL[pix];
        }
        st.T[p] = Tf;
        st.DS[p] = Tf * (st.d[p].x * bg.x + st.d[p].y * bg.y + st.d[p].z * bg.z - st.d[p].w);
        mx = max(mx, st.my_last[p]);
    }
    return mx;
}

// Back-to-front walk of nl staged slots of a batch (slot j holds entry b_end - 1 - j of the tile's
// run): list[0..nl) (in slot order, from band_list) with band_cull, else j0 .. j0 + nl - 1, for
// this thread's P pixels, adding the per-Gaussian record gradients. The live state comes by
// reference: T, DS per pixel (for even P as pixel pairs T2, DS2 instead) and the pixels'
// dL/dRGBA (d; for even P also as pairs DX2, DY2, DZ2). Every lane of a warp calls it with the
// same slots (the walk holds warp-wide votes).
template <int P, int H = (P / 2 > 0 ? P / 2 : 1)>
__device__ __forceinline__ void bwd_batch(const unsigned char* list, int j0, int nl, int b_end, float fx,
                                          float fyg, int q0, float (&T)[P], float (&DS)[P], const float4 (&d)[P],
                                          const unsigned (&my_last)[P], F2 (&T2)[H], F2 (&DS2)[H],
                                          const F2 (&DX2)[H], const F2 (&DY2)[H], const F2 (&DZ2)[H],
                                          const float4* s_a, const float4* s_b, const float2* s_c,
                                          const long long* s_gi, float4* __restrict__ g0, float4* __restrict__ g1,
                                          float* __restrict__ g2) {
    constexpr int NG = (P + 3) / 4;  // 4-row exponent groups a thread spans
    const int lane = threadIdx.x & 31;
    if constexpr (P == 1) {
        // One pixel per thread: kBwdSteps1 list entries per step, their exponents and reach tests
        // first, then the chain-rule updates in walk order, then the entries' record gradients,
        // so that the dependent chains of the entries (shared loads, exponent, ex2, the reductions
        // and atomics) overlap; lone warps of the heaviest tiles are latency-bound (two entries
        // per step: the 800^2 view 0.541 -> 0.521 ms; the 10k-Gaussian 128^2 view 0.091 ->
        // 0.081 ms). Per pixel the same operations in the same order as the path below.
        // The chain rule of one entry for the thread's pixel (as the odd-P path below):
        auto chain = [&](const float4& bb, float blue, const RowGroup& rgq, float p2, bool ok, float (&vv)[8],
                         float& vb, auto clamp) {
            constexpr bool CLAMP = decltype(clamp)::value;
            const float G = fast_ex2(p2);
            const float raw = bb.y * G;
            const float alpha = CLAMP ? fminf(kAlphaMax, raw) : raw;
            const float r = fast_rcp(1.0f - alpha);
            const float Ti = T[0] * r;
            const float w = ok ? Ti * alpha : 0.0f;
            const float4 dd = d[0];
            vv[6] = fmaf(w, dd.x, vv[6]);
            vv[7] = fmaf(w, dd.y, vv[7]);
            vb = fmaf(w, dd.z, vb);
            const float dc = dd.x * bb.z + dd.y * bb.w + dd.z * blue;
            const float dalpha = Ti * dc - DS[0] * r;
            DS[0] = fmaf(w, dc, DS[0]);
            T[0] = ok ? Ti : T[0];
            const bool live = CLAMP ? ok && raw < kAlphaMax : ok;
            const float dP = live ? dalpha * raw : 0.0f;
            vv[5] += live ? dalpha * G : 0.0f;
            const float dxp = rgq.dx, dyp = rgq.dy0 - (float)(q0 & 3);
            const float px_ = dP * dxp, py_ = dP * dyp;
            vv[0] += px_;
            vv[1] += py_;
            vv[2] = fmaf(px_, dxp, vv[2]);
            vv[3] = fmaf(px_, dyp, vv[3]);
            vv[4] = fmaf(py_, dyp, vv[4]);
        };
        // the record gradients of one entry (as below)
        auto emit = [&](const float4& a, const float4& bb, int j, const float (&vv)[8], float vb, bool contrib) {
            const unsigned m = __ballot_sync(0xffffffffu, contrib);
            if (m == 0u) return;
            const long long gi = s_gi[j];
            float* t0 = reinterpret_cast<float*>(g0 + gi);
            float* t1 = reinterpret_cast<float*>(g1 + gi);
            const float il = 2.0f / kLog2e;
            const float tm = fmaf(a.w, vv[0], vv[1]);
            if (__popc(m) <= kDirectLanes) {
                if (contrib) {
                    const float du = fmaf(bb.x, vv[0], a.z * a.w * tm) * il;
                    const float dv = a.z * tm * il;
                    atomicAdd(reinterpret_cast<float4*>(t0), make_float4(du, dv, -0.5f * vv[2], -vv[3]));
                    atomicAdd(reinterpret_cast<float4*>(t1), make_float4(-0.5f * vv[4], vv[5], vv[6], vv[7]));
                    atomicAdd(&g2[gi], vb);
                }
            } else {
                const float tv[8] = {fmaf(bb.x, vv[0], a.z * a.w * tm) * il, a.z * tm * il,
                                     -0.5f * vv[2], -vv[3], -0.5f * vv[4], vv[5], vv[6], vv[7]};
                const float x = warp_sum8_transposed(tv, lane);
                const float vbs = warp_sum(vb);
                const int idx = lane >> 2;
                if ((lane & 3) == 0) atomicAdd(idx < 4 ? t0 + idx : t1 + (idx - 4), x);
                if (lane == 0) atomicAdd(&g2[gi], vbs);
            }
        };
        for (int i = 0; i < nl; i += kBwdSteps1) {
            float4 aq[kBwdSteps1], bq[kBwdSteps1];
            float2 cq[kBwdSteps1];
            RowGroup rq[kBwdSteps1];
            float pq[kBwdSteps1];
            bool okq[kBwdSteps1];
            int jq[kBwdSteps1];
            bool any = false;
#pragma unroll
            for (int k = 0; k < kBwdSteps1; ++k) {
                const bool has = i + k < nl;
                const int ii = has ? i + k : i;  // past the end: a repeat of entry i, never in reach
                jq[k] = band_cull<P>() ? (int)list[ii] : j0 + ii;
                aq[k] = s_a[jq[k]];
                bq[k] = s_b[jq[k]];
                cq[k] = s_c[jq[k]];
                rq[k] = row_group(aq[k], bq[k], fx, fyg);
                pq[k] = row_p2(rq[k], aq[k], q0 & 3);
                okq[k] = has && b_end - 1 - jq[k] < (int)my_last[0] && in_reach(pq[k], cq[k].y);
                any = any || okq[k];
            }
            if (!__any_sync(0xffffffffu, any)) continue;
            float vq[kBwdSteps1][8], vbq[kBwdSteps1];
#pragma unroll
            for (int k = 0; k < kBwdSteps1; ++k) {
#pragma unroll
                for (int m = 0; m < 8; ++m) vq[k][m] = 0.f;
                vbq[k] = 0.f;
                if (bq[k].y > kNoClampOpacity)
                    chain(bq[k], cq[k].x, rq[k], pq[k], okq[k], vq[k], vbq[k], std::true_type{});
                else
                    chain(bq[k], cq[k].x, rq[k], pq[k], okq[k], vq[k], vbq[k], std::false_type{});
            }
#pragma unroll
            for (int k = 0; k < kBwdSteps1; ++k) emit(aq[k], bq[k], jq[k], vq[k], vbq[k], okq[k]);
        }
    } else {
        for (int i = 0; i < nl; ++i) {
            const int j = band_cull<P>() ? (int)list[i] : j0 + i;
            const int ee = b_end - 1 - j;
            const float4 a = s_a[j];
            const float4 bb = s_b[j];
            const float2 cc = s_c[j];
            const float blue = cc.x;
            // per-thread sums over its pixels: vv = (m1, m2, m3, m4, m5, d o', d r, d g) with the
            // moments m1 = sum dP dx, m2 = sum dP dy, m3 = sum dP dx^2, m4 = sum dP dx dy,
            // m5 = sum dP dy^2 (the conic and mean gradients are linear in them); vb = d blue
            float vv[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            float vb = 0.f;
            float p2[P];
            bool ok0[P];
            bool any = false;
            RowGroup rgp[NG];  // every aligned group of 4 rows has its own base, whatever P is
#pragma unroll
            for (int gq = 0; gq < NG; ++gq) rgp[gq] = row_group(a, bb, fx, fyg + 4.0f * (float)gq);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                p2[p] = row_p2(rgp[(q0 + p) >> 2], a, (q0 + p) & 3);
                ok0[p] = ee < (int)my_last[p] && in_reach(p2[p], cc.y);
                any = any || ok0[p];
            }
            if (!__any_sync(0xffffffffu, any)) continue;
            bool contrib = false;
            // the pixels' chain rule, instantiated with and without the 0.99 clamp (a uniform branch
            // on the entry's o': at or below kNoClampOpacity, alpha = o' G and dalpha/dP = o' G)
            auto pixels = [&](auto clamp) {
                constexpr bool CLAMP = decltype(clamp)::value;
                if constexpr (P % 2 == 0) {
                    // pixel pairs in paired float32 arithmetic (the same IEEE operations per pixel; only
                    // the order in which a thread adds its pixels' moments differs)
                    const F2 zero = f2(0.f, 0.f), one = f2(1.f, 1.f);
                    const F2 O2 = f2(bb.y, bb.y), BZ = f2(bb.z, bb.z), BW = f2(bb.w, bb.w), BL = f2(blue, blue);
                    F2 V0 = zero, V1 = zero, V2 = zero, V3 = zero, V4 = zero, V5 = zero, V6 = zero, V7 = zero;
                    F2 VB = zero;
#pragma unroll
                    for (int h = 0; h < P / 2; ++h) {
                        const int pa = 2 * h, pb = 2 * h + 1;
                        const F2 G = f2(fast_ex2(p2[pa]), fast_ex2(p2[pb]));
                        const F2 RAW = mul2(O2, G);
                        float raw_a, raw_b;
                        split(RAW, raw_a, raw_b);
                        const float al_a = CLAMP ? fminf(kAlphaMax, raw_a) : raw_a;
                        const float al_b = CLAMP ? fminf(kAlphaMax, raw_b) : raw_b;
                        const bool ok_a = ok0[pa], ok_b = ok0[pb];
                        contrib = contrib || ok_a || ok_b;
                        const F2 A = f2(al_a, al_b);
                        float om_a, om_b;
                        split(sub2(one, A), om_a, om_b);
                        const F2 R = f2(fast_rcp(om_a), fast_rcp(om_b));
                        const F2 TI = mul2(T2[h], R);
                        F2 TN;  // T in front of the entry: recovered for a contributor, unchanged otherwise
                        {
                            float ti_a, ti_b, t_a, t_b;
                            split(TI, ti_a, ti_b);
                            split(T2[h], t_a, t_b);
                            TN = f2(ok_a ? ti_a : t_a, ok_b ? ti_b : t_b);
                        }
                        // the weight T_i alpha_i as T_i - T_{i+1} (0 for a skipped pixel), so that one select
                        // serves both; it differs from the rounded product by the rounding of T_i, under
                        // 2^-24 T_i / alpha_i, relative 1.5e-5 at the cut-off
                        const F2 W = sub2(TN, T2[h]);
                        V6 = fma2(W, DX2[h], V6);
                        V7 = fma2(W, DY2[h], V7);
                        VB = fma2(W, DZ2[h], VB);
                        const F2 DC = fma2(DZ2[h], BL, fma2(DY2[h], BW, mul2(DX2[h], BZ)));  // dL/dC . c_i
                        const F2 DA = sub2(mul2(TI, DC), mul2(DS2[h], R));                    // dL/dalpha
                        DS2[h] = fma2(W, DC, DS2[h]);
                        T2[h] = TN;
                        // dalpha/dP = o' G while unclamped, 0 on the 0.99 clamp and for skipped pixels
                        // (selected after the product, so that an infinite G never reaches the sums)
                        const bool live_a = CLAMP ? ok_a && raw_a < kAlphaMax : ok_a;
                        const bool live_b = CLAMP ? ok_b && raw_b < kAlphaMax : ok_b;
                        float dp_a, dp_b, dg_a, dg_b;
                        split(mul2(DA, RAW), dp_a, dp_b);
                        split(mul2(DA, G), dg_a, dg_b);
                        const F2 DP = f2(live_a ? dp_a : 0.0f, live_b ? dp_b : 0.0f);
                        V5 = add2(V5, f2(live_a ? dg_a : 0.0f, live_b ? dg_b : 0.0f));
                        const RowGroup& ga = rgp[(q0 + pa) >> 2];
                        const RowGroup& gb = rgp[(q0 + pb) >> 2];
                        const F2 DXP = f2(ga.dx, gb.dx);
                        const F2 DYP = f2(ga.dy0 - (float)((q0 + pa) & 3), gb.dy0 - (float)((q0 + pb) & 3));
                        const F2 PX = mul2(DP, DXP), PY = mul2(DP, DYP);
                        V0 = add2(V0, PX);
                        V1 = add2(V1, PY);
                        V2 = fma2(PX, DXP, V2);
                        V3 = fma2(PX, DYP, V3);
                        V4 = fma2(PY, DYP, V4);
                    }
                    const F2 Vs[8] = {V0, V1, V2, V3, V4, V5, V6, V7};
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        float lo, hi;
                        split(Vs[k], lo, hi);
                        vv[k] = lo + hi;
                    }
                    float lo, hi;
                    split(VB, lo, hi);
                    vb = lo + hi;
                } else {
                    // the P pixels update independently (predicated, no branches) so they interleave
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        const float G = fast_ex2(p2[p]);
                        const float raw = bb.y * G;
                        const float alpha = CLAMP ? fminf(kAlphaMax, raw) : raw;
                        const bool ok = ok0[p];
                        contrib = contrib || ok;
                        const float r = fast_rcp(1.0f - alpha);
                        const float Ti = T[p] * r;
                        const float w = ok ? Ti * alpha : 0.0f;
                        const float4 dd = d[p];
                        vv[6] = fmaf(w, dd.x, vv[6]);
                        vv[7] = fmaf(w, dd.y, vv[7]);
                        vb = fmaf(w, dd.z, vb);
                        const float dc = dd.x * bb.z + dd.y * bb.w + dd.z * blue;  // dL/dC . c_i
                        const float dalpha = Ti * dc - DS[p] * r;
                        DS[p] = fmaf(w, dc, DS[p]);
                        T[p] = ok ? Ti : T[p];
                        // dalpha/dP = o' G while unclamped, 0 on the 0.99 clamp (and for skipped pixels,
                        // selected rather than multiplied so that an infinite G never reaches the sums)
                        const bool live = CLAMP ? ok && raw < kAlphaMax : ok;
                        const float dP = live ? dalpha * raw : 0.0f;
                        vv[5] += live ? dalpha * G : 0.0f;
                        const float dxp = rgp[(q0 + p) >> 2].dx, dyp = rgp[(q0 + p) >> 2].dy0 - (float)((q0 + p) & 3);
                        const float px_ = dP * dxp, py_ = dP * dyp;
                        vv[0] += px_;
                        vv[1] += py_;
                        vv[2] = fmaf(px_, dxp, vv[2]);
                        vv[3] = fmaf(px_, dyp, vv[3]);
                        vv[4] = fmaf(py_, dyp, vv[4]);
                    }
                }
            };
            if (bb.y > kNoClampOpacity) pixels(std::true_type{});
            else pixels(std::false_type{});
            const unsigned m = __ballot_sync(0xffffffffu, contrib);
            if (m == 0u) continue;
            const long long gi = s_gi[j];
            float* t0 = reinterpret_cast<float*>(g0 + gi);
            float* t1 = reinterpret_cast<float*>(g1 + gi);
            // moments -> (du, dv, da, db, dc): P = p2 / log2(e), p2 = C' (dy + beta dx)^2 + G' dx^2
            //   (staged C' = a.z, beta = a.w, G' = bb.x), so with t = beta m1 + m2
            //   du = 2 (G' m1 + C' beta t)/log2e, dv = 2 C' t/log2e,
            //   da = -m3/2, db = -m4, dc = -m5/2
            const float il = 2.0f / kLog2e;
            const float tm = fmaf(a.w, vv[0], vv[1]);
            if (__popc(m) <= kDirectLanes) {  // few contributing lanes: each adds its own, no reduction
                if (contrib) {
                    const float du = fmaf(bb.x, vv[0], a.z * a.w * tm) * il;
                    const float dv = a.z * tm * il;
                    atomicAdd(reinterpret_cast<float4*>(t0), make_float4(du, dv, -0.5f * vv[2], -vv[3]));
                    atomicAdd(reinterpret_cast<float4*>(t1), make_float4(-0.5f * vv[4], vv[5], vv[6], vv[7]));
                    atomicAdd(&g2[gi], vb);
                }
            } else {
                // every lane turns its moments into (du, dv, da, db, dc) first (linear, so the sum
                // is the same): no lane-dependent branches after the reduction
                const float tv[8] = {fmaf(bb.x, vv[0], a.z * a.w * tm) * il, a.z * tm * il,
                                     -0.5f * vv[2], -vv[3], -0.5f * vv[4], vv[5], vv[6], vv[7]};
                const float x = warp_sum8_transposed(tv, lane);  // lane holds the total of index lane >> 2
                vb = warp_sum(vb);
                const int idx = lane >> 2;
                if ((lane & 3) == 0) atomicAdd(idx < 4 ? t0 + idx : t1 + (idx - 4), x);
                if (lane == 0) atomicAdd(&g2[gi], vb);
            }
        }
    }
}

// Stages entry e of the tile's run (record values[run0 + e] of view base vbase) in slot `slot`,
// with its record index for the gradient atomics.
__device__ __forceinline__ void stage_entry_bwd(int slot, int e, const float2* __restrict__ xy,
                                                const float4* __restrict__ conic_o, const float4* __restrict__ rgbd,
                                                long long n, const unsigned* __restrict__ values, unsigned run0,
                                                long long vbase, float4* s_a, float4* s_b, float2* s_c,
                                                long long* s_gi, float2* s_rows) {
    const unsigned g = values[run0 + e];
    long long gi = vbase + g;
    float4 sa, sb;
    float2 sc;
    if (g < (unsigned long long)n) {
        stage_gaussian(xy[gi], conic_o[gi], rgbd[gi], sa, sb, sc);
    } else {  // never for a completed sort; a zero-opacity stand-in keeps reads in bounds
        gi = vbase;
        stage_gaussian(make_float2(0.f, 0.f), make_float4(1.f, 0.f, 1.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f), sa,
                       sb, sc);
    }
    s_a[slot] = sa;
    s_b[slot] = sb;
    s_c[slot] = sc;
    s_gi[slot] = gi;
    if (s_rows != nullptr) s_rows[slot] = reach_rows(sa, sb, sc);
}

// Back-to-front walk of the entries [e_lo, e_top) of a tile's run for this thread's P pixels
// from their state, adding the per-Gaussian record gradients; e_top is at most the CTA's largest
// last contributor and w_top the warp's (entries at or beyond it are skipped by the whole warp).
// e_lo and e_top are the same for every thread of the CTA.
template <int P, int TH>
__device__ __forceinline__ void bwd_walk(int e_lo, int e_top, int w_top, const float2* __restrict__ xy,
                                         const float4* __restrict__ conic_o, const float4* __restrict__ rgbd,
                                         long long n, const unsigned* __restrict__ values, unsigned run0,
                                         long long vbase, float fx, float fyg, int q0, float ylo, BwdPix<P>& st,
                                         float4* s_a, float4* s_b, float2* s_c, long long* s_gi, float2* s_rows,
                                         unsigned char* list, float4* __restrict__ g0, float4* __restrict__ g1,
                                         float* __restrict__ g2) {
    constexpr int NT = kTile * TH / P;
    float T[P], DS[P];
    float4 d[P];
    unsigned my_last[P];
    F2 T2[P / 2 > 0 ? P / 2 : 1], DS2[P / 2 > 0 ? P / 2 : 1];  // even P: the same, as pixel pairs
    F2 DX2[P / 2 > 0 ? P / 2 : 1], DY2[P / 2 > 0 ? P / 2 : 1], DZ2[P / 2 > 0 ? P / 2 : 1];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        T[p] = st.T[p];
        DS[p] = st.DS[p];
        d[p] = st.d[p];
        my_last[p] = st.my_last[p];
    }
    if constexpr (P % 2 == 0) {
#pragma unroll
        for (int h = 0; h < P / 2; ++h) {
            T2[h] = f2(T[2 * h], T[2 * h + 1]);
            DS2[h] = f2(DS[2 * h], DS[2 * h + 1]);
            DX2[h] = f2(d[2 * h].x, d[2 * h + 1].x);
            DY2[h] = f2(d[2 * h].y, d[2 * h + 1].y);
            DZ2[h] = f2(d[2 * h].z, d[2 * h + 1].z);
        }
    }
    for (int b_end = e_top; b_end > e_lo; b_end -= kBwdBatch) {
        const int b_start = max(e_lo, b_end - kBwdBatch);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kBwdBatch / NT; ++q) {
            const int slot = threadIdx.x + q * NT;
            const int e = b_end - 1 - slot;
            if (e >= b_start)
                stage_entry_bwd(slot, e, xy, conic_o, rgbd, n, values, run0, vbase, s_a, s_b, s_c, s_gi,
                                band_cull<P>() ? s_rows : nullptr);
        }
        __syncthreads();
        // entries at or beyond every lane's last contributor are skipped by the whole warp, and with
        // band_cull so are those out of reach of the warp's rows
        const int j0 = max(0, b_end - w_top);
        int nl = b_end - b_start - j0;
        if constexpr (band_cull<P>()) nl = band_list(j0, b_end - b_start, ylo, ylo + (float)(2 * P - 1), s_rows, list);
        bwd_batch<P>(list, j0, nl, b_end, fx, fyg, q0, T, DS, d, my_last, T2, DS2, DX2, DY2, DZ2, s_a, s_b, s_c, s_gi,
                     g0, g1, g2);
    }
}

// Per tile, P vertically adjacent pixels per thread; each warp covers a compact band of rows.
// With 4 pixels per thread on 16-pixel-high tiles the register budget is set for 18 CTAs per SM
// (56 registers), two more than the compiler's own choice.
template <int P, int TH>
__global__ void __launch_bounds__(kTile * TH / P, P == 4 && TH == 16 ? 18 : 1) k_render_bwd(
    const float2* __restrict__ xy, const float4* __restrict__ conic_o, const float4* __restrict__ rgbd, long long n,
    const unsigned* __restrict__ values, const uint2* __restrict__ ranges, const __grid_constant__ CamBatch cb,
    float3 bg, const float* __restrict__ final_T, const unsigned* __restrict__ last_in,
    const float4* __restrict__ dL, float4* __restrict__ g0, float4* __restrict__ g1, float* __restrict__ g2,
    int split_min) {
    __shared__ float4 s_a[kBwdBatch];
    __shared__ float4 s_b[kBwdBatch];
    __shared__ float2 s_c[kBwdBatch];
    __shared__ long long s_gi[kBwdBatch];
    __shared__ float2 s_rows[band_cull<P>() ? kBwdBatch : 1];
    __shared__ unsigned char s_list[band_cull<P>() ? kTile * TH / P / 32 * kBwdBatch : 1];
    __shared__ unsigned s_max;
    const long long tile = blockIdx.x;
    const int v = view_of_tile(cb, tile);
    const CamDev& cam = cb.c[v];
    const int local = (int)(tile - cam.tile0);
    const int tx = local % cam.gx, ty = local / cam.gx;
    const int px = tx * kTile + (threadIdx.x & (kTile - 1));
    const int py0 = ty * TH + (threadIdx.x / kTile) * P;
    const float fx = (float)px + 0.5f;
    // offset of this thread's first row in its 4-row group (0 whenever P is a multiple of 4,
    // since py0 is then one too: known at compile time, so the groups are indexed statically)
    const int q0 = (P % 4 == 0) ? 0 : (py0 & 3);
    const float fyg = (float)(py0 - q0) + 0.5f;            // centre of the group's first row
    const uint2 rg = ranges[tile];
    BwdPix<P> st;
    const unsigned mx = bwd_init<P>(cam, px, py0, bg, final_T, last_in, dL, st);
    if (threadIdx.x == 0) s_max = 0u;
    __syncthreads();
    atomicMax(&s_max, mx);
    __syncthreads();
    const int top = (int)s_max;
    // tile selection as in k_render: split_min >= 0 keeps the walks of at most split_min entries,
    // split_min < 0 the walks longer than -split_min - 1
    const int len = min((int)(rg.y - rg.x), top);
    if (split_min >= 0 ? len > split_min : len <= -split_min - 1) return;
    const float ylo = (float)(py0 - ((int)(threadIdx.x & 16u) >> 4) * P) + 0.5f;  // this warp's first pixel row
    bwd_walk<P, TH>(0, top, (int)__reduce_max_sync(0xffffffffu, mx), xy, conic_o, rgbd, n, values, rg.x,
                (long long)v * n, fx, fyg, q0, ylo, st, s_a, s_b, s_c, s_gi, s_rows,
                s_list + (band_cull<P>() ? (threadIdx.x >> 5) * kBwdBatch : 0), g0, g1, g2);
}

// ---------------------------------------------------------------------------------------------
// Split backward for tiles with long runs: a cluster of kSplit CTAs per tile, CTA k walking the
// chunk [lo_k, hi_k) of the run back to front (the chunks as in the split forward). Each chunk
// needs the transmittance just behind its part of the walk and DS, the colour accumulated
// behind it dotted with dL/dC. Both follow from per-chunk forward partials over the pixel's
// contributors (entries before its last contributor): T_k = prod (1 - alpha) and
// D_k = dL/dC . sum T_local alpha c (from T_local = 1). With T_pre_k = prod_{j<k} T_j, the chunk
// walks back from T_pre_k T_k (from T_final in the chunk holding the last contributor) and
// DS = T_final (dL/dC . bg - dL/dA) + sum_{j>k} T_pre_j D_j. The partials travel through
// distributed shared memory. Only walks longer than split_min entries are split; k_render_bwd,
// launched after, takes every other tile.
// ---------------------------------------------------------------------------------------------
// Forward partials of the entries [lo, hi) over each pixel's contributors (entries before its
// last contributor with alpha >= 1/255): T_k and D_k as above. lo, hi uniform per CTA.
template <int P, int TH>
__device__ __forceinline__ void bwd_chunk_partial(int lo, int hi, const float2* __restrict__ xy,
                                                  const float4* __restrict__ conic_o, const float4* __restrict__ rgbd,
                                                  long long n, const unsigned* __restrict__ values, unsigned run0,
                                                  long long vbase, float fx, float fyg, int q0, const BwdPix<P>& st,
                                                  float (&Tk)[P], float (&Dk)[P], float4* s_a, float4* s_b,
                                                  float2* s_c) {
    constexpr int NT = kTile * TH / P;
    constexpr int NG = (P + 3) / 4;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        Tk[p] = 1.0f;
        Dk[p] = 0.0f;
    }
    for (int b0 = lo; b0 < hi; b0 += kBwdBatch) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kBwdBatch / NT; ++q) {
            const int slot = threadIdx.x + q * NT;
            const int e = b0 + slot;
            if (e < hi) {
                const unsigned g = values[run0 + e];
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
        const int cnt = min(kBwdBatch, hi - b0);
        for (int j = 0; j < cnt; ++j) {
            const int e = b0 + j;
            const float4 a = s_a[j];
            const float4 bb = s_b[j];
            const float2 cc = s_c[j];
            RowGroup rgp[NG];
#pragma unroll
            for (int gq = 0; gq < NG; ++gq) rgp[gq] = row_group(a, bb, fx, fyg + 4.0f * (float)gq);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float p2 = row_p2(rgp[(q0 + p) >> 2], a, (q0 + p) & 3);
                const bool ok = e < (int)st.my_last[p] && in_reach(p2, cc.y);
                const float alpha = fminf(kAlphaMax, bb.y * fast_ex2(p2));
                const bool add = ok;
                const float w = add ? alpha * Tk[p] : 0.0f;
                const float4 dd = st.d[p];
                Dk[p] = fmaf(w, dd.x * bb.z + dd.y * bb.w + dd.z * cc.x, Dk[p]);
                Tk[p] = add ? Tk[p] * (1.0f - alpha) : Tk[p];  // the forward's T (1 - alpha)
            }
        }
    }
}

template <int P, int TH>
__global__ void __cluster_dims__(kSplit, 1, 1) __launch_bounds__(kTile * TH / P) k_render_bwd_split(
    const float2* __restrict__ xy, const float4* __restrict__ conic_o, const float4* __restrict__ rgbd, long long n,
    const unsigned* __restrict__ values, const uint2* __restrict__ ranges, const __grid_constant__ CamBatch cb,
    float3 bg, int split_min, const float* __restrict__ final_T, const unsigned* __restrict__ last_in,
    const float4* __restrict__ dL, float4* __restrict__ g0, float4* __restrict__ g1, float* __restrict__ g2) {
    __shared__ float4 s_a[kBwdBatch];
    __shared__ float4 s_b[kBwdBatch];
    __shared__ float2 s_c[kBwdBatch];
    __shared__ long long s_gi[kBwdBatch];
    __shared__ float2 s_rows[band_cull<P>() ? kBwdBatch : 1];
    __shared__ unsigned char s_list[band_cull<P>() ? kTile * TH / P / 32 * kBwdBatch : 1];
    __shared__ float s_T[kTile * TH], s_D[kTile * TH];
    __shared__ unsigned s_max;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const long long tile = blockIdx.x / kSplit;
    const int v = view_of_tile(cb, tile);
    const CamDev& cam = cb.c[v];
    const int local = (int)(tile - cam.tile0);
    const int tx = local % cam.gx, ty = local / cam.gx;
    const int px = tx * kTile + (threadIdx.x & (kTile - 1));
    const int py0 = ty * TH + (threadIdx.x / kTile) * P;
    const float fx = (float)px + 0.5f;
    const int q0 = (P % 4 == 0) ? 0 : (py0 & 3);
    const float fyg = (float)(py0 - q0) + 0.5f;
    const uint2 rg = ranges[tile];
    const long long vbase = (long long)v * n;
    BwdPix<P> st;
    const unsigned mx = bwd_init<P>(cam, px, py0, bg, final_T, last_in, dL, st);
    if (threadIdx.x == 0) s_max = 0u;
    __syncthreads();
    atomicMax(&s_max, mx);
    __syncthreads();
    const int cta_last = (int)s_max, warp_last = (int)__reduce_max_sync(0xffffffffu, mx);
    int nc, lo, hi;
    split_chunk(min((int)(rg.y - rg.x), cta_last), split_min, rank, nc, lo, hi);
    if (nc == 1) return;  // a short walk: k_render_bwd takes it (the whole cluster leaves, before any cluster barrier)
    int pl[P];  // pixel index within the tile
#pragma unroll
    for (int p = 0; p < P; ++p) pl[p] = (threadIdx.x / kTile) * P * kTile + p * kTile + (threadIdx.x & (kTile - 1));
    // 1. per-chunk forward partials (one chunk: not needed)
    float Tk[P], Dk[P];
    if (nc > 1 && rank < nc) {
        bwd_chunk_partial<P, TH>(lo, hi, xy, conic_o, rgbd, n, values, rg.x, vbase, fx, fyg, q0, st, Tk, Dk, s_a, s_b,
                                 s_c);
    } else {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            Tk[p] = 1.0f;
            Dk[p] = 0.0f;
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
        s_T[pl[p]] = Tk[p];
        s_D[pl[p]] = Dk[p];
    }
    cl.sync();
    // 2. the state just behind this chunk's part of the walk
    if (nc > 1 && rank < nc) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            float t = 1.0f, behind = 0.0f, tpre = 1.0f;
            for (int j = 0; j < nc; ++j) {
                const float Tj = *cl.map_shared_rank(&s_T[pl[p]], j);
                if (j == rank) tpre = t;
                if (j > rank) behind = fmaf(t, *cl.map_shared_rank(&s_D[pl[p]], j), behind);
                t *= Tj;
            }
            const int last = (int)st.my_last[p];
            if (last > lo && last <= hi) {  // the chunk holding the last contributor: behind it, T_final
                // (st.T, st.DS as initialised)
            } else if (last > hi) {
                st.T[p] = tpre * Tk[p];
                st.DS[p] += behind;
            }
        }
    }
    cl.sync();  // every CTA has read the partials it needs
    // 3. walk back over the chunk
    if (rank < nc) {
        const int top = min(hi, cta_last);
        const float ylo = (float)(py0 - ((int)(threadIdx.x & 16u) >> 4) * P) + 0.5f;
        bwd_walk<P, TH>(lo, top, min(hi, warp_last), xy, conic_o, rgbd, n, values, rg.x, vbase, fx, fyg, q0, ylo, st,
                        s_a, s_b, s_c, s_gi, s_rows, s_list + (band_cull<P>() ? (threadIdx.x >> 5) * kBwdBatch : 0),
                        g0, g1, g2);
    }
}

// ------------------------------------------------------------------------- a7
template <int PREC, bool SH>
__global__ void __launch_bounds__(256, 2) k_project_bwd(const ivrgs_gaussians g, const float* __restrict__ table,
                                                     const __grid_constant__ CamBatch cb, float lowpass,
                                                     const float4* __restrict__ g0, const float4* __restrict__ g1,
                                                     const float* __restrict__ g2, const ivrgs_gaussians grad,
                                                     float* __restrict__ egrad, int accumulate) {
    __shared__ float s_red[8][8];
    __shared__ int s_model;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = g.n;
    const bool active = i < n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int M = g.n_models;
    GaussLocal G;
    if (active) load_gauss<PREC>(g, table, M, i, G);
    else G.visible = false;
    if constexpr (!SH) G.sh = nullptr;  // the instantiation without SH colour carries none of its code
    const bool tl_on = __ldg(table + (long long)M * IVRGS_EDIT_STRIDE + 11) != 0.0f;  // uniform
    float dmu[3] = {0.f, 0.f, 0.f}, dSl[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // dSl: dL/dSigma in the Gaussian's frame
    float dcv[3] = {0.f, 0.f, 0.f}, dkp[4] = {0.f, 0.f, 0.f, 0.f}, dnn[3] = {0.f, 0.f, 0.f}, dop = 0.f;
    // the next view's record gradients are loaded before this view's arithmetic (latency overlap)
    float4 na = make_float4(0.f, 0.f, 0.f, 0.f), nbq = na;
    float nbl = 0.f;
    if (G.visible && cb.n > 0) {
        na = g0[i];
        nbq = g1[i];
        nbl = g2[i];
    }
    for (int v = 0; v < cb.n; ++v) {
        const CamDev& c = cb.c[v];
        float dlv[3] = {0.f, 0.f, 0.f};
        const float4 a = na, b = nbq;
        const float bl = nbl;
        if (G.visible && v + 1 < cb.n) {
            const long long o1 = (long long)(v + 1) * n + i;
            na = g0[o1];
            nbq = g1[o1];
            nbl = g2[o1];
        }
        if (G.visible) {
            const bool any = (a.x != 0.f) | (a.y != 0.f) | (a.z != 0.f) | (a.w != 0.f) | (b.x != 0.f) |
                             (b.y != 0.f) | (b.z != 0.f) | (b.w != 0.f) | (bl != 0.f);
            ViewLocal V;
            if (any) project_view(G, c, lowpass, V);
            if (SH && any && V.visible && G.sh) {  // ---- 3DGS colour: SH coefficients and the view direction
                dop += b.y;
                const float Gr[3] = {b.z, b.w, bl};
                const float sx = -V.vd[0], sy = -V.vd[1], sz = -V.vd[2];
                const int nb = (G.sh_deg + 1) * (G.sh_deg + 1);
                float* gsh = grad.sh + i * 3ll * nb;
                const float gr0 = V.shc[0] ? 0.f : Gr[0], gr1 = V.shc[1] ? 0.f : Gr[1], gr2 = V.shc[2] ? 0.f : Gr[2];
                float dd[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    if (t >= nb) break;
                    float gx, gy, gz;
                    const float Yt = sh_term(t, sx, sy, sz, gx, gy, gz);
                    gsh[3 * t + 0] += gr0 * Yt;
                    gsh[3 * t + 1] += gr1 * Yt;
                    gsh[3 * t + 2] += gr2 * Yt;
                    const float w = gr0 * __ldg(G.sh + 3 * t) + gr1 * __ldg(G.sh + 3 * t + 1) + gr2 * __ldg(G.sh + 3 * t + 2);
                    dd[0] += w * gx;
                    dd[1] += w * gy;
                    dd[2] += w * gz;
                }
                // d = (mu - campos) / |mu - campos|
                const float pd = sx * dd[0] + sy * dd[1] + sz * dd[2];
                const float iv = 1.0f / V.vlen;
                dmu[0] += (dd[0] - sx * pd) * iv;
                dmu[1] += (dd[1] - sy * pd) * iv;
                dmu[2] += (dd[2] - sz * pd) * iv;
            }
            if (any && V.visible) {
                if (!G.sh) {
                dop += b.y;
                // ---- shading
                const float Gr[3] = {b.z, b.w, bl};
                const float Gc = Gr[0] * G.cv[0] + Gr[1] * G.cv[1] + Gr[2] * G.cv[2];
                const float Gs = Gr[0] + Gr[1] + Gr[2];
                const float kd = G.kp[0] + G.kp[1] * V.nl;
                for (int k = 0; k < 3; ++k) dcv[k] += kd * Gr[k];
                dkp[0] += Gc;
                dkp[1] += V.nl * Gc;
                float dnh = 0.f;
                if (V.gate) {
                    dkp[2] += Gs * V.spow;
                    dkp[3] += Gs * G.kp[2] * V.spow * logf(V.nh);
                    dnh = Gs * G.kp[2] * G.kp[3] * V.spow / V.nh;
                }
                const float dnl = G.kp[1] * Gc;
                const float snl = V.ndl > 0.f ? 1.f : (V.ndl < 0.f ? -1.f : 0.f);
                const float snh = V.ndh > 0.f ? 1.f : (V.ndh < 0.f ? -1.f : 0.f);
                float dl[3], dh[3], dv[3] = {0.f, 0.f, 0.f};
                for (int k = 0; k < 3; ++k) {
                    dnn[k] += dnl * snl * V.l[k] + dnh * snh * V.h[k];
                    dl[k] = dnl * snl * G.nn[k];
                    dh[k] = dnh * snh * G.nn[k];
                }
                if (V.hlen > 0.f) {
                    const float hd = V.h[0] * dh[0] + V.h[1] * dh[1] + V.h[2] * dh[2];
                    const float ih = 1.0f / V.hlen;
                    for (int k = 0; k < 3; ++k) {
                        const float t = (dh[k] - V.h[k] * hd) * ih;
                        dv[k] += t;
                        dl[k] += t;
                    }
                }
                if (c.headlight) {
                    for (int k = 0; k < 3; ++k) dv[k] += dl[k];
                } else {  // gradient w.r.t. the direction used: the table's global light or the view's
                    const float* lh = G.tl_on ? G.tl : c.light;
                    const float ll = G.tl_on ? G.tl_len : c.light_len;
                    const float ld = lh[0] * dl[0] + lh[1] * dl[1] + lh[2] * dl[2];
                    for (int k = 0; k < 3; ++k) dlv[k] = (dl[k] - lh[k] * ld) / ll;
                }
                {
                    const float vd = V.vd[0] * dv[0] + V.vd[1] * dv[1] + V.vd[2] * dv[2];
                    const float iv = 1.0f / V.vlen;
                    for (int k = 0; k < 3; ++k) dmu[k] -= (dv[k] - V.vd[k] * vd) * iv;
                }
                }
                // ---- conic -> Sigma' -> (Sigma, T), in the eigenbasis of Sigma'
                // dL/dSigma' = -K Gk K, K = Sigma'^-1 (the conic), Gk = dL/dK as a symmetric
                // matrix. With Sigma' = E diag(l1, l2) E^T this is E D E^T, D_ij = -(E^T Gk E)_ij
                // k_i k_j, where k1 = 1/l1 and k2 = l1/det are the conic's eigenvalues. Written out
                // in the pixel basis (the adjugate over det^2), the long-axis entry of a long, thin
                // Gaussian is a difference of terms larger by (l1/l2)^2; here each entry of D is
                // one product. dSigma is kept in the Gaussian's own frame, Rq^T dSigma Rq = P^T D P
                // with P = E^T T Rq, where the long axis's row of P is nearly orthogonal to the
                // short one's, so the scale gradients need no cancellation either.
                const float A = V.A, B = V.B, C = V.C;
                const float hd = 0.5f * (A - C);
                const float rr = sqrtf(hd * hd + B * B);
                const float l1 = 0.5f * (A + C) + rr;
                // e1 from the row of (Sigma' - l1 I) whose entries do not cancel; e2 = (-ey, ex)
                float ex = hd >= 0.f ? hd + rr : B, ey = hd >= 0.f ? B : rr - hd;
                const float en = ex * ex + ey * ey;
                if (en > 0.f) {
                    const float sn = rsqrtf(en);
                    ex *= sn;
                    ey *= sn;
                } else {
                    ex = 1.f;
                    ey = 0.f;
                }
                const float ga = a.z, gb = a.w, gc = b.x;  // dL/d(a, b, c) of the conic
                const float H11 = ga * ex * ex + gb * ex * ey + gc * ey * ey;
                const float H22 = ga * ey * ey - gb * ex * ey + gc * ex * ex;
                const float H12 = (gc - ga) * ex * ey + 0.5f * gb * (ex * ex - ey * ey);
                const float k1 = 1.0f / l1, k2 = l1 / V.det;
                const float D11 = -H11 * k1 * k1, D12 = -H12 * (k1 * k2), D22 = -H22 * k2 * k2;
                const float* T = V.T;
                float p1[3], p2[3];  // rows of P = E^T T Rq
                {
                    float q1[3], q2[3];
                    for (int j = 0; j < 3; ++j) {
                        q1[j] = ex * T[j] + ey * T[3 + j];
                        q2[j] = ex * T[3 + j] - ey * T[j];
                    }
                    for (int k = 0; k < 3; ++k) {
                        p1[k] = q1[0] * G.Rq[k] + q1[1] * G.Rq[3 + k] + q1[2] * G.Rq[6 + k];
                        p2[k] = q2[0] * G.Rq[k] + q2[1] * G.Rq[3 + k] + q2[2] * G.Rq[6 + k];
                    }
                }
                // dSigma in the Gaussian's frame += P^T D P (xx, xy, xz, yy, yz, zz)
                {
                    int o = 0;
                    for (int r = 0; r < 3; ++r)
                        for (int k = r; k < 3; ++k, ++o)
                            dSl[o] += D11 * p1[r] * p1[k] + D12 * (p1[r] * p2[k] + p2[r] * p1[k]) + D22 * p2[r] * p2[k];
                }
                // dT = 2 dSigma' T Sigma = 2 E D (P diag(s^2)) Rq^T
                float dT[6];
                {
                    float w1[3], w2[3];
                    for (int k = 0; k < 3; ++k) {
                        const float s2 = G.sc[k] * G.sc[k];
                        const float a1 = p1[k] * s2, a2 = p2[k] * s2;
                        w1[k] = D11 * a1 + D12 * a2;
                        w2[k] = D12 * a1 + D22 * a2;
                    }
                    for (int j = 0; j < 3; ++j) {
                        const float u1 = w1[0] * G.Rq[3 * j] + w1[1] * G.Rq[3 * j + 1] + w1[2] * G.Rq[3 * j + 2];
                        const float u2 = w2[0] * G.Rq[3 * j] + w2[1] * G.Rq[3 * j + 1] + w2[2] * G.Rq[3 * j + 2];
                        dT[j] = 2.f * (ex * u1 - ey * u2);
                        dT[3 + j] = 2.f * (ey * u1 + ex * u2);
                    }
                }
                // dJ = dT W^T; only J00, J02, J11, J12 are non-zero
                const float dJ00 = dT[0] * c.R[0] + dT[1] * c.R[1] + dT[2] * c.R[2];
                const float dJ02 = dT[0] * c.R[6] + dT[1] * c.R[7] + dT[2] * c.R[8];
                const float dJ11 = dT[3] * c.R[3] + dT[4] * c.R[4] + dT[5] * c.R[5];
                const float dJ12 = dT[3] * c.R[6] + dT[4] * c.R[7] + dT[5] * c.R[8];
                const float iz = V.iz, iz2 = iz * iz;
                float dmc[3] = {0.f, 0.f, 0.f};
                dmc[2] += dJ00 * (-c.fx * iz2) + dJ11 * (-c.fy * iz2);
                if (V.clx) {
                    dmc[2] += dJ02 * (c.fx * V.txc * iz2);
                } else {
                    dmc[0] += dJ02 * (-c.fx * iz2);
                    dmc[2] += dJ02 * (2.f * c.fx * V.x * iz2 * iz);
                }
                if (V.cly) {
                    dmc[2] += dJ12 * (c.fy * V.tyc * iz2);
                } else {
                    dmc[1] += dJ12 * (-c.fy * iz2);
                    dmc[2] += dJ12 * (2.f * c.fy * V.y * iz2 * iz);
                }
                // mean2D: u = fx x/z + cx
                dmc[0] += a.x * c.fx * iz;
                dmc[1] += a.y * c.fy * iz;
                dmc[2] += -(a.x * c.fx * V.x + a.y * c.fy * V.y) * iz2;
                for (int k = 0; k < 3; ++k) dmu[k] += c.R[k] * dmc[0] + c.R[3 + k] * dmc[1] + c.R[6 + k] * dmc[2];
            }
        }
        if (!c.headlight) {  // uniform across the grid: per-view light gradient, block-reduced
            float r0 = warp_sum(dlv[0]), r1 = warp_sum(dlv[1]), r2 = warp_sum(dlv[2]);
            __syncthreads();
            if (lane == 0) { s_red[warp][0] = r0; s_red[warp][1] = r1; s_red[warp][2] = r2; }
            __syncthreads();
            if (threadIdx.x < 3) {
                float t = 0.f;
                for (int w = 0; w < 8; ++w) t += s_red[w][threadIdx.x];
                // the table's global light (its slot) or the view's light_dir (the per-view tail)
                const long long slot = tl_on ? (long long)M * IVRGS_EDIT_STRIDE + 8
                                             : (long long)M * IVRGS_EDIT_STRIDE + 12 + 4 * v;
                if (t != 0.f) atomicAdd(&egrad[slot + threadIdx.x], t);
            }
        }
    }
    // ---- view-independent chains
    float dlam[4] = {0.f, 0.f, 0.f, 0.f}, dbias[4] = {0.f, 0.f, 0.f, 0.f};
    float dcp[3] = {0.f, 0.f, 0.f}, dsm = 0.f;
    if (active) {
        float gm[3] = {0.f, 0.f, 0.f}, gls[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f}, gn[3] = {0.f, 0.f, 0.f};
        float glogit = 0.f, gdc[3] = {0.f, 0.f, 0.f}, gk[4] = {0.f, 0.f, 0.f, 0.f};
        if (G.visible) {
            for (int k = 0; k < 3; ++k) gm[k] = dmu[k];
            // Sigma = Rq diag(s^2) Rq^T with dSigma given in the Gaussian's frame (dSl = Rq^T dSigma Rq):
            // d log s_k = 2 s_k^2 dSl_kk, dL/dRq = 2 Rq dSl diag(s^2)
            const float dS[9] = {dSl[0], dSl[1], dSl[2], dSl[1], dSl[3], dSl[4], dSl[2], dSl[4], dSl[5]};
            float dR[9];
            for (int k = 0; k < 3; ++k) {
                const float s2 = G.sc[k] * G.sc[k];
                gls[k] = 2.f * s2 * dS[4 * k];
                for (int r = 0; r < 3; ++r)
                    dR[3 * r + k] = 2.f * s2 * (G.Rq[3 * r] * dS[k] + G.Rq[3 * r + 1] * dS[3 + k] + G.Rq[3 * r + 2] * dS[6 + k]);
            }
            const float w = G.qn[0], x = G.qn[1], y = G.qn[2], z = G.qn[3];
            float dq[4];
            dq[0] = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
            dq[1] = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] -
                           2.f * x * dR[8]);
            dq[2] = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] -
                           2.f * y * dR[8]);
            dq[3] = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] + y * dR[5] +
                           x * dR[6] + y * dR[7]);
            const float qd = w * dq[0] + x * dq[1] + y * dq[2] + z * dq[3];
            for (int k = 0; k < 4; ++k) gq[k] = (dq[k] - G.qn[k] * qd) / G.qlen;
            const float nd = G.nn[0] * dnn[0] + G.nn[1] * dnn[1] + G.nn[2] * dnn[2];
            for (int k = 0; k < 3; ++k) gn[k] = (dnn[k] - G.nn[k] * nd) / G.nlen;
            glogit = dop * G.sm * G.sig * (1.f - G.sig);
            dsm = dop * G.sig;
            const float* lam = table + (long long)M * IVRGS_EDIT_STRIDE;
            for (int k = 0; k < 4; ++k) {
                gk[k] = __ldg(lam + k) * dkp[k];
                dlam[k] = G.k[k] * dkp[k];
                dbias[k] = dkp[k];
            }
            for (int k = 0; k < 3; ++k) {
                gdc[k] = dcv[k];
                dcp[k] = dcv[k];
            }
        }
        float* gmn = static_cast<float*>(grad.mean);
        float* gsc = static_cast<float*>(grad.log_scale);
        float* gco = static_cast<float*>(grad.dcolor);
        float* gno = static_cast<float*>(grad.normal);
        float4* gqu = static_cast<float4*>(grad.quat);
        float4* gka = static_cast<float4*>(grad.kads);
        float* glo = static_cast<float*>(grad.opacity_logit);
        if (accumulate) {  // add to the gradients of earlier view waves
            for (int k = 0; k < 3; ++k) {
                gm[k] += gmn[3 * i + k];
                gls[k] += gsc[3 * i + k];
                gdc[k] += gco[3 * i + k];
                gn[k] += gno[3 * i + k];
            }
            const float4 a4 = gqu[i], b4 = gka[i];
            gq[0] += a4.x; gq[1] += a4.y; gq[2] += a4.z; gq[3] += a4.w;
            gk[0] += b4.x; gk[1] += b4.y; gk[2] += b4.z; gk[3] += b4.w;
            glogit += glo[i];
        }
        for (int k = 0; k < 3; ++k) {
            gmn[3 * i + k] = gm[k];
            gsc[3 * i + k] = gls[k];
            gco[3 * i + k] = gdc[k];
            gno[3 * i + k] = gn[k];
        }
        gqu[i] = make_float4(gq[0], gq[1], gq[2], gq[3]);
        gka[i] = make_float4(gk[0], gk[1], gk[2], gk[3]);
        glo[i] = glogit;
    }
    // ---- edit gradients: global lambda, b block-reduced; per-model terms warp-reduced when the warp is
    // uniform in its model (composed models are contiguous), else per lane
    {
        float r[8];
        for (int k = 0; k < 4; ++k) { r[k] = warp_sum(dlam[k]); r[4 + k] = warp_sum(dbias[k]); }
        __syncthreads();
        if (lane == 0)
            for (int k = 0; k < 8; ++k) s_red[warp][k] = r[k];
        __syncthreads();
        if (threadIdx.x < 8) {
            float t = 0.f;
            for (int w = 0; w < 8; ++w) t += s_red[w][threadIdx.x];
            if (t != 0.f) atomicAdd(&egrad[(long long)M * IVRGS_EDIT_STRIDE + threadIdx.x], t);
        }
    }
    {
        const int model = active ? G.model : -1;
        // a block of one model (the usual case) adds its per-model sums with one atomic each: with
        // one atomic per warp, a single-model scene (the 500k-Gaussian view) put 15,600 atomics on
        // each of the same four words (k_project_bwd 0.066 ms)
        if (threadIdx.x == 0) s_model = model;
        __syncthreads();
        const int m0 = s_model;
        if (__syncthreads_and(model == m0)) {
            const float r0 = warp_sum(dcp[0]), r1 = warp_sum(dcp[1]), r2 = warp_sum(dcp[2]), r3 = warp_sum(dsm);
            if (lane == 0) { s_red[warp][0] = r0; s_red[warp][1] = r1; s_red[warp][2] = r2; s_red[warp][3] = r3; }
            __syncthreads();
            if (threadIdx.x < 4 && m0 >= 0) {
                float t = 0.f;
                for (int w = 0; w < 8; ++w) t += s_red[w][threadIdx.x];
                if (t != 0.f) atomicAdd(egrad + (long long)m0 * IVRGS_EDIT_STRIDE + threadIdx.x, t);
            }
            return;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, model);
        if (peers == 0xffffffffu) {
            float r0 = warp_sum(dcp[0]), r1 = warp_sum(dcp[1]), r2 = warp_sum(dcp[2]), r3 = warp_sum(dsm);
            if (lane == 0 && model >= 0) {
                float* eg = egrad + (long long)model * IVRGS_EDIT_STRIDE;
                if (r0 != 0.f) atomicAdd(eg + 0, r0);
                if (r1 != 0.f) atomicAdd(eg + 1, r1);
                if (r2 != 0.f) atomicAdd(eg + 2, r2);
                if (r3 != 0.f) atomicAdd(eg + 3, r3);
            }
        } else if (model >= 0) {
            float* eg = egrad + (long long)model * IVRGS_EDIT_STRIDE;
            if (dcp[0] != 0.f) atomicAdd(eg + 0, dcp[0]);
            if (dcp[1] != 0.f) atomicAdd(eg + 1, dcp[1]);
            if (dcp[2] != 0.f) atomicAdd(eg + 2, dcp[2]);
            if (dsm != 0.f) atomicAdd(eg + 3, dsm);
        }
    }
}

cudaError_t launch_render_backward(const ivrgs_gaussians* g, const float* table, const ivrgs_projected* p,
                                   const ivrgs_bins* b, const CamBatch& cb, float lowpass, const float* bg,
                                   const float* final_T, const uint32_t* last, const float* dL, char* ws,
                                   ivrgs_gaussians* grad, float* edit_grad, int accumulate, cudaStream_t s) {
    const long long vn = p->n * (long long)cb.n;
    float4* g0 = reinterpret_cast<float4*>(ws);
    float4* g1 = g0 + vn;
    float* g2 = reinterpret_cast<float*>(g1 + vn);
    cudaError_t e;
    if ((e = cudaMemsetAsync(ws, 0, (size_t)vn * 36, s)) != cudaSuccess) return e;
    const long long ne = (long long)g->n_models * IVRGS_EDIT_STRIDE + 12 + 4ll * cb.n;
    // the per-view light gradients (the tail) always start at zero; the edit gradients only
    // when not accumulating over view waves
    const long long ne0 = accumulate ? (long long)g->n_models * IVRGS_EDIT_STRIDE + 12 : 0;
    if ((e = cudaMemsetAsync(edit_grad + ne0, 0, sizeof(float) * (size_t)(ne - ne0), s)) != cudaSuccess) return e;
    if (cb.n_tiles > 0) {
        IVRGS_PROF("k_render_bwd", s);
        const float2* xy = reinterpret_cast<const float2*>(p->xy);
        const float4* co = reinterpret_cast<const float4*>(p->conic_o);
        const float4* cd = reinterpret_cast<const float4*>(p->rgbd);
        const uint2* rg = reinterpret_cast<const uint2*>(b->ranges);
        const float3 bgc = make_float3(bg[0], bg[1], bg[2]);
        const float4* dl = reinterpret_cast<const float4*>(dL);
        const int ppt = blend_ppt(options().render_bwd_ppt, cb.n_tiles, true);
        // with the split walk, walks longer than split_min go to the cluster kernel, on a side
        // stream beside k_render_bwd, which takes the rest; without it, k_render_bwd takes every tile
        const bool split = use_split(options().render_split, cb.n_tiles);
        const int sm = split ? options().render_split_min : INT_MAX;
        cudaStream_t side = s;
        if (split && (e = split_fork(s, &side)) != cudaSuccess) return e;
        if (split && options().render_split == 4) {  // the long walks first, on the side stream, unsplit
            const int hs = -sm - 1;
            blend_shape(ppt, cb.th, [&](auto P, auto TH) {
                constexpr int kP = decltype(P)::value, kTH = decltype(TH)::value;
                k_render_bwd<kP, kTH><<<(unsigned)cb.n_tiles, kTile * kTH / kP, 0, side>>>(
                    xy, co, cd, p->n, b->values, rg, cb, bgc, final_T, last, dl, g0, g1, g2, hs);
            });
        } else if (split) {
            const unsigned grid = (unsigned)(cb.n_tiles * kSplit);
            blend_shape(ppt, cb.th, [&](auto P, auto TH) {
                constexpr int kP = decltype(P)::value, kTH = decltype(TH)::value;
                k_render_bwd_split<kP, kTH><<<grid, kTile * kTH / kP, 0, side>>>(
                    xy, co, cd, p->n, b->values, rg, cb, bgc, sm, final_T, last, dl, g0, g1, g2);
            });
        }
        blend_shape(ppt, cb.th, [&](auto P, auto TH) {
            constexpr int kP = decltype(P)::value, kTH = decltype(TH)::value;
            k_render_bwd<kP, kTH><<<(unsigned)cb.n_tiles, kTile * kTH / kP, 0, s>>>(
                xy, co, cd, p->n, b->values, rg, cb, bgc, final_T, last, dl, g0, g1, g2, sm);
        });
        if (split) {
            const cudaError_t el = cudaGetLastError();
            const cudaError_t ej = split_join(s);
            if (el != cudaSuccess) return el;
            if (ej != cudaSuccess) return ej;
        }
    }
    return launch_project_backward(g, table, cb, lowpass, g0, g1, g2, grad, edit_grad, accumulate, s);
}

cudaError_t launch_project_backward(const ivrgs_gaussians* g, const float* table, const CamBatch& cb, float lowpass,
                                    const float4* g0, const float4* g1, const float* g2, ivrgs_gaussians* grad,
                                    float* edit_grad, int accumulate, cudaStream_t s) {
    cudaError_t e;
    if (g->sh && !accumulate && g->n > 0) {  // SH gradients are added view by view
        const size_t nb = (size_t)(g->sh_degree + 1) * (g->sh_degree + 1);
        if ((e = cudaMemsetAsync(grad->sh, 0, sizeof(float) * 3 * nb * (size_t)g->n, s)) != cudaSuccess) return e;
    }
    if (g->n > 0) {
        IVRGS_PROF("k_project_bwd", s);
        const unsigned nb = (unsigned)((g->n + 255) / 256);
#define IVRGS_PBWD(P, S) k_project_bwd<P, S><<<nb, 256, 0, s>>>(*g, table, cb, lowpass, g0, g1, g2, *grad, edit_grad, accumulate)
        if (g->sh) {
            if (g->precision == IVRGS_VQ) IVRGS_PBWD(IVRGS_VQ, true);
            else if (g->precision == IVRGS_MIXED) IVRGS_PBWD(IVRGS_MIXED, true);
            else IVRGS_PBWD(IVRGS_FP32, true);
        } else {
            if (g->precision == IVRGS_VQ) IVRGS_PBWD(IVRGS_VQ, false);
            else if (g->precision == IVRGS_MIXED) IVRGS_PBWD(IVRGS_MIXED, false);
            else IVRGS_PBWD(IVRGS_FP32, false);
        }
#undef IVRGS_PBWD
    }
    return cudaGetLastError();
}

}  // namespace ivrgs

// Per-tile front-to-back compositing (row a5; Sec. 3 second equation).
//
// One CTA per 16x16 tile; each of its 256/P threads owns P vertically adjacent pixels of one
// column, so every Gaussian staged in shared memory is read once per P pixels and the P
// transmittance chains run interleaved; a warp covers a compact band of 32P/16 rows, so a
// Gaussian that misses the band lets the whole warp skip it. The tile's sorted run is walked in batches of 256
// Gaussians: the CTA stages each batch (mean, conic pre-scaled by -log2(e)/2 so that the
// exponent is one FMA chain, opacity, colour), then every pixel walks it. The CTA leaves as
// soon as every pixel has reached T < 1e-4 (barrier count).
#include <climits>
#include <type_traits>
#include <cooperative_groups.h>

#include "blend_alpha.cuh"

namespace cg = cooperative_groups;

namespace ivrgs {

constexpr int kBatch = 256;
constexpr int kSteps1 = 4;  // list entries per step of the one-pixel walk (1, 2, 4 or 8)

// Per-thread state of P vertically adjacent pixels of one column of a tile.
template <int P>
struct FwdPix {
    float C0[P], C1[P], C2[P], T[P];
    unsigned last[P];
    bool done[P];
};

// Front-to-back walk of the staged entries [j0, j1) of a batch whose first entry is entry b0 of
// the tile's run, for this thread's P pixels, from their current state. Every lane of a warp
// calls it with the same j0, j1 (the walk holds warp-wide votes); list is the warp's scratch
// for the slots it walks. `last` records 1 + the position of the last added entry in the run.
template <int P>
__device__ __forceinline__ void fwd_batch(int j0, int j1, int b0, const TilePos& tp, FwdPix<P>& s,
                                          const float4* s_a, const float4* s_b, const float2* s_c,
                                          const float2* s_rows, unsigned char* list) {
    constexpr int NG = (P + 3) / 4;  // 4-row exponent groups a thread spans
    // with band_cull, only the slots whose reach rows meet this warp's rows (the others are out
    // of reach of every pixel of the warp, which in_reach would decide entry by entry)
    int nl = j1 - j0;
    if constexpr (band_cull<P>()) {
        const float ylo = (float)(tp.py0 - ((int)(threadIdx.x & 16u) >> 4) * P) + 0.5f;
        nl = band_list(j0, j1, ylo, ylo + (float)(2 * P - 1), s_rows, list);
    }
    if constexpr (P == 1) {
        // One pixel per thread: kSteps1 list entries per step, all their exponents, reach tests
        // and exponentials first, then the updates in order, so that a warp's chains of dependent
        // operations per entry (shared loads, exponent, ex2) overlap. At one pixel per thread a
        // warp is the whole walk of its two rows, and on a view whose heaviest tiles set the
        // launch time the lone warps that still run are latency-bound: on the 800^2 view the
        // heaviest tile alone on an SM takes 374 / 325 / 276 us at 1 / 2 / 4 entries per step, the
        // launch 0.437 / 0.410 / 0.362 ms (62 registers at 4, so 4 CTAs per SM instead of 6: the
        // shorter chains win all the same). The same operations per pixel in the same order as
        // below, so the same bits.
        auto one = [&](bool ok, const float4& bb, const float2& cc, float G, unsigned idx, auto clamp) {
            const float Tn = __fmul_rn(s.T[0], one_minus_alpha<decltype(clamp)::value>(bb.y, G));
            const bool stop = ok && Tn < kTMin;
            const bool add = ok && !stop;
            const float Tk = add ? Tn : s.T[0];
            const float w = s.T[0] - Tk;
            s.C0[0] = fmaf(w, bb.z, s.C0[0]);
            s.C1[0] = fmaf(w, bb.w, s.C1[0]);
            s.C2[0] = fmaf(w, cc.x, s.C2[0]);
            s.T[0] = Tk;
            s.last[0] = add ? idx : s.last[0];
            s.done[0] = s.done[0] || stop;
        };
        for (int i = 0; i < nl; i += kSteps1) {
            float4 bq[kSteps1];
            float2 cq[kSteps1];
            float pq[kSteps1];
            bool okq[kSteps1];
            int jq[kSteps1];
            bool any = false;
#pragma unroll
            for (int k = 0; k < kSteps1; ++k) {
                const bool has = i + k < nl;
                const int ii = has ? i + k : i;  // past the end: a repeat of entry i, never in reach
                jq[k] = band_cull<P>() ? (int)list[ii] : j0 + ii;
                const float4 aq = s_a[jq[k]];
                bq[k] = s_b[jq[k]];
                cq[k] = s_c[jq[k]];
                pq[k] = row_p2(row_group(aq, bq[k], tp.fx, tp.fyg), aq, tp.q0);
                okq[k] = has && !s.done[0] && in_reach(pq[k], cq[k].y);
                any = any || okq[k];
            }
            if (__any_sync(0xffffffffu, any)) {
                float gq[kSteps1];
#pragma unroll
                for (int k = 0; k < kSteps1; ++k) gq[k] = fast_ex2(pq[k]);
#pragma unroll
                for (int k = 0; k < kSteps1; ++k) {
                    const bool ok = okq[k] && !s.done[0];  // an earlier entry may have ended the pixel
                    const unsigned idx = (unsigned)(b0 + jq[k] + 1);
                    if (bq[k].y > kNoClampOpacity) one(ok, bq[k], cq[k], gq[k], idx, std::true_type{});
                    else one(ok, bq[k], cq[k], gq[k], idx, std::false_type{});
                }
            }
            if ((i & 7) + kSteps1 >= 8 && __all_sync(0xffffffffu, s.done[0])) break;  // every 8 entries
        }
    } else {
        // the entries in groups of 8, the termination vote after each group (no per-entry test of
        // the position in the group: 0.715 -> 0.702 ms on the 1M-Gaussian, 8-view workload)
        for (int i0 = 0; i0 < nl; i0 += 8) {
            const int i1 = min(nl, i0 + 8);
            for (int i = i0; i < i1; ++i) {
                const int j = band_cull<P>() ? (int)list[i] : j0 + i;
                const float4 a = s_a[j];
                const float4 bb = s_b[j];
                const float2 cc = s_c[j];
                float p2[P];
                bool ok[P];
                bool any = false;
                RowGroup rgp[NG];  // every aligned group of 4 rows has its own base, whatever P is
#pragma unroll
                for (int gq = 0; gq < NG; ++gq) rgp[gq] = row_group(a, bb, tp.fx, tp.fyg + 4.0f * (float)gq);
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    p2[p] = row_p2(rgp[(tp.q0 + p) >> 2], a, (tp.q0 + p) & 3);
                    ok[p] = !s.done[p] && in_reach(p2[p], cc.y);
                    any = any || ok[p];
                }
                if (__any_sync(0xffffffffu, any)) {
                    const unsigned idx = (unsigned)(b0 + j + 1);
                    // the P pixels update independently (predicated, no branches) so they interleave;
                    // instantiated with and without the 0.99 clamp (a uniform branch on the entry's o')
                    auto update = [&](auto clamp) {
#pragma unroll
                        for (int p = 0; p < P; ++p) {
                            const float Tn =
                                __fmul_rn(s.T[p], one_minus_alpha<decltype(clamp)::value>(bb.y, fast_ex2(p2[p])));
                            const bool stop = ok[p] && Tn < kTMin;
                            const bool add = ok[p] && !stop;
                            // the weight T alpha as the drop of T (exact: Sterbenz), so that one select
                            // serves both; it differs from the rounded product T alpha by the rounding of
                            // T (1 - alpha), at most 2^-24 T per entry, under 1.6e-5 in all (T falls by
                            // 1/255 at least per entry)
                            const float Tk = add ? Tn : s.T[p];
                            const float w = s.T[p] - Tk;
                            s.C0[p] = fmaf(w, bb.z, s.C0[p]);
                            s.C1[p] = fmaf(w, bb.w, s.C1[p]);
                            s.C2[p] = fmaf(w, cc.x, s.C2[p]);
                            s.T[p] = Tk;
                            s.last[p] = add ? idx : s.last[p];
                            s.done[p] = s.done[p] || stop;
                        }
                    };
                    if (bb.y > kNoClampOpacity) update(std::true_type{});
                    else update(std::false_type{});
                }
            }
            bool mine = true;
#pragma unroll
            for (int p = 0; p < P; ++p) mine = mine && s.done[p];
            if (__all_sync(0xffffffffu, mine)) break;
        }
    }
}

// Stages entry e of the tile's run (record values[run0 + e] of view base vbase) in slot `slot`.
__device__ __forceinline__ void stage_entry(int slot, int e, const float2* __restrict__ xy,
                                            const float4* __restrict__ conic_o, const float4* __restrict__ rgbd,
                                            long long n, const unsigned* __restrict__ values, unsigned run0,
                                            long long vbase, float4* s_a, float4* s_b, float2* s_c,
                                            float2* s_rows) {
    const unsigned g = values[run0 + e];
    float4 sa, sb;
    float2 sc;
    if (g < (unsigned long long)n) {
        const long long gi = vbase + g;
        stage_gaussian(xy[gi], conic_o[gi], rgbd[gi], sa, sb, sc);
    } else {  // never for a completed sort; a zero-opacity stand-in keeps reads in bounds
        stage_gaussian(make_float2(0.f, 0.f), make_float4(1.f, 0.f, 1.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f), sa,
                       sb, sc);
    }
    s_a[slot] = sa;
    s_b[slot] = sb;
    s_c[slot] = sc;
    if (s_rows != nullptr) s_rows[slot] = reach_rows(sa, sb, sc);
}

// Front-to-back walk of the entries [e0, e1) of a tile's run for this thread's P pixels, from
// their current state. The CTA stages batches of kBatch Gaussians in shared memory and leaves
// as soon as every pixel is done (barrier count), so e0, e1 must be the same for every thread
// of the CTA.
template <int P, int TH>
__device__ __forceinline__ void fwd_walk(int e0, int e1, const float2* __restrict__ xy,
                                         const float4* __restrict__ conic_o, const float4* __restrict__ rgbd,
                                         long long n, const unsigned* __restrict__ values, unsigned run0,
                                         long long vbase, const TilePos& tp, FwdPix<P>& s, float4* s_a, float4* s_b,
                                         float2* s_c, float2* s_rows, unsigned char* s_list) {
    constexpr int NT = kTile * TH / P;
    for (int b0 = e0; b0 < e1; b0 += kBatch) {
        bool all = true;
#pragma unroll
        for (int p = 0; p < P; ++p) all = all && s.done[p];
        if (__syncthreads_count(all) == NT) break;
#pragma unroll
        for (int q = 0; q < kBatch / NT; ++q) {
            const int slot = threadIdx.x + q * NT;
            const int e = b0 + slot;
            if (e < e1)
                stage_entry(slot, e, xy, conic_o, rgbd, n, values, run0, vbase, s_a, s_b, s_c,
                            band_cull<P>() ? s_rows : nullptr);
        }
        __syncthreads();
        // the walk below holds warp-wide votes: a warp skips or leaves it only as a whole
        if (__all_sync(0xffffffffu, all)) continue;
        unsigned char* list = s_list + (band_cull<P>() ? (threadIdx.x >> 5) * kBatch : 0);  // this warp's
        fwd_batch<P>(0, min(kBatch, e1 - b0), b0, tp, s, s_a, s_b, s_c, s_rows, list);
    }
}

template <int P, int TH>
__global__ void __launch_bounds__(kTile * TH / P) k_render(const float2* __restrict__ xy,
                                                         const float4* __restrict__ conic_o,
                                                         const float4* __restrict__ rgbd, long long n,
                                                         const unsigned* __restrict__ values,
                                                         const uint2* __restrict__ ranges,
                                                         const __grid_constant__ CamBatch cb, float3 bg,
                                                         float4* __restrict__ rgba, float* __restrict__ final_T,
                                                         unsigned* __restrict__ last_out, int split_min) {
    __shared__ float4 s_a[kBatch];
    __shared__ float4 s_b[kBatch];
    __shared__ float2 s_c[kBatch];
    __shared__ float2 s_rows[band_cull<P>() ? kBatch : 1];
    __shared__ unsigned char s_list[band_cull<P>() ? kTile * TH / P / 32 * kBatch : 1];
    const long long tile = blockIdx.x;
    const uint2 rg = ranges[tile];
    // tile selection: split_min >= 0 keeps the runs of at most split_min entries (the others go
    // to k_render_split, or to a launch of their own), split_min < 0 the runs longer than
    // -split_min - 1
    const int len = (int)(rg.y - rg.x);
    if (split_min >= 0 ? len > split_min : len <= -split_min - 1) return;
    const int v = view_of_tile(cb, tile);
    const CamDev& cam = cb.c[v];
    const TilePos tp = tile_pos<P, TH>(cam, tile);
    FwdPix<P> s;
    bool inside[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        inside[p] = tp.px < cam.W && tp.py0 + p < cam.H;
        s.C0[p] = s.C1[p] = s.C2[p] = 0.f;
        s.T[p] = 1.f;
        s.last[p] = 0;
        s.done[p] = !inside[p];
    }
    fwd_walk<P, TH>(0, (int)(rg.y - rg.x), xy, conic_o, rgbd, n, values, rg.x, (long long)v * n, tp, s, s_a, s_b, s_c,
                s_rows, s_list);
#pragma unroll
    for (int p = 0; p < P; ++p)
        if (inside[p]) {
            const long long pix = cam.pix0 + (long long)(tp.py0 + p) * cam.W + tp.px;
            rgba[pix] = make_float4(s.C0[p] + s.T[p] * bg.x, s.C1[p] + s.T[p] * bg.y, s.C2[p] + s.T[p] * bg.z,
                                    1.0f - s.T[p]);
            final_T[pix] = s.T[p];
            last_out[pix] = s.last[p];
        }
}

// ---------------------------------------------------------------------------------------------
// Split walk for tiles with long runs (the run of a tile is one serial chain per pixel; on a
// view whose few hundred heavy tiles carry most of the entries, the heaviest tile's chain sets the
// launch time). A thread-block cluster of kSplit CTAs takes one tile; CTA k composites the
// chunk [k ch, (k + 1) ch) of the run from T = 1, so the chunks run on kSplit SMs at once.
// Front-to-back "over" is associative: with per-chunk colour C_k and transmittance T_k, the
// pixel is sum_k T_pre_k C_k, T_pre_k = prod_{j<k} T_j. The one coupling is the termination at
// T < 1e-4, which depends on the transmittance in front of the chunk: a chunk whose pixel walk
// stopped on its own (T_k fell below 1e-4 from 1) or whose T_pre_k T_k is below 1e-4 holds the
// pixel's termination; that chunk is walked again from T_pre_k with the sequential rule (exact
// termination entry and last contributor), and the chunks behind it are dropped. The partial
// results travel through distributed shared memory. Only runs longer than split_min entries
// are split: their clusters are the only ones that stay, and k_render, launched after, walks
// every other tile (a cluster per light tile would hold 8 CTA slots for one CTA's work).
// Products regroup, so T can differ from the sequential walk in the last bits (a termination
// decision only at a float32 near-tie).
// ---------------------------------------------------------------------------------------------
template <int P, int TH>
__global__ void __cluster_dims__(kSplit, 1, 1) __launch_bounds__(kTile * TH / P)
    k_render_split(const float2* __restrict__ xy, const float4* __restrict__ conic_o, const float4* __restrict__ rgbd,
                   long long n, const unsigned* __restrict__ values, const uint2* __restrict__ ranges,
                   const __grid_constant__ CamBatch cb, float3 bg, int split_min, float4* __restrict__ rgba,
                   float* __restrict__ final_T, unsigned* __restrict__ last_out) {
    __shared__ float4 s_a[kBatch];
    __shared__ float4 s_b[kBatch];
    __shared__ float2 s_c[kBatch];
    __shared__ float2 s_rows[band_cull<P>() ? kBatch : 1];
    __shared__ unsigned char s_list[band_cull<P>() ? kTile * TH / P / 32 * kBatch : 1];
    constexpr int NPIX = kTile * TH;
    __shared__ float s_T[NPIX], s_C0[NPIX], s_C1[NPIX], s_C2[NPIX];
    __shared__ unsigned s_last[NPIX];
    __shared__ int s_state[NPIX];  // after the walk: 1 stopped in the chunk; after the merge: 0 dropped,
                                       // 1 passed, 2 holds the termination
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const long long tile = blockIdx.x / kSplit;
    const int v = view_of_tile(cb, tile);
    const CamDev& cam = cb.c[v];
    const TilePos tp = tile_pos<P, TH>(cam, tile);
    const uint2 rg = ranges[tile];
    const long long vbase = (long long)v * n;
    int nc, lo, hi;
    split_chunk((int)(rg.y - rg.x), split_min, rank, nc, lo, hi);
    if (nc == 1) return;  // a short run: k_render walks it (the whole cluster leaves, before any cluster barrier)
    const bool active = rank < nc;
    FwdPix<P> s;
    bool inside[P];
    int pl[P];  // pixel index within the tile
#pragma unroll
    for (int p = 0; p < P; ++p) {
        inside[p] = tp.px < cam.W && tp.py0 + p < cam.H;
        pl[p] = (threadIdx.x / kTile) * P * kTile + p * kTile + (threadIdx.x & (kTile - 1));
        s.C0[p] = s.C1[p] = s.C2[p] = 0.f;
        s.T[p] = 1.f;
        s.last[p] = 0;
        s.done[p] = !inside[p];
    }
    // 1. every active CTA walks its chunk from T = 1 (CTA 0's walk is the sequential one)
    if (active) fwd_walk<P, TH>(lo, hi, xy, conic_o, rgbd, n, values, rg.x, vbase, tp, s, s_a, s_b, s_c, s_rows, s_list);
#pragma unroll
    for (int p = 0; p < P; ++p) {
        s_T[pl[p]] = s.T[p];
        s_state[pl[p]] = (inside[p] && s.done[p]) ? 1 : 0;
    }
    cl.sync();
    // 2. transmittance in front of this chunk and whether an earlier chunk holds the termination
    float Tpre[P];
    int state[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        float t = 1.0f;
        bool ended = false;
        for (int j = 0; j < rank && j < nc; ++j) {
            const float Tj = *cl.map_shared_rank(&s_T[pl[p]], j);
            const int stop_j = *cl.map_shared_rank(&s_state[pl[p]], j);
            if (!ended) {
                if (stop_j || t * Tj < kTMin) ended = true;
                else t *= Tj;
            }
        }
        Tpre[p] = t;
        if (!active || ended || !inside[p]) state[p] = 0;
        else if (rank > 0 && (s.done[p] || t * s.T[p] < kTMin)) state[p] = 2;
        else state[p] = 1;
    }
    cl.sync();  // every CTA has read the chunk results it needs
    // 3. the chunk holding a pixel's termination is walked again from T_pre (sequential rule)
    bool rewalk = false;
#pragma unroll
    for (int p = 0; p < P; ++p) rewalk = rewalk || state[p] == 2;
    if (__syncthreads_or(rewalk)) {
        FwdPix<P> r;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            r.C0[p] = r.C1[p] = r.C2[p] = 0.f;
            r.T[p] = Tpre[p];
            r.last[p] = 0;
            r.done[p] = state[p] != 2;
        }
        fwd_walk<P, TH>(lo, hi, xy, conic_o, rgbd, n, values, rg.x, vbase, tp, r, s_a, s_b, s_c, s_rows, s_list);
#pragma unroll
        for (int p = 0; p < P; ++p)
            if (state[p] == 2) {
                s.C0[p] = r.C0[p];
                s.C1[p] = r.C1[p];
                s.C2[p] = r.C2[p];
                s.T[p] = r.T[p];
                s.last[p] = r.last[p];
            }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const bool scale = state[p] == 1 && rank > 0;  // a passed chunk's colour seen through T_pre
        s_C0[pl[p]] = state[p] == 0 ? 0.f : (scale ? Tpre[p] * s.C0[p] : s.C0[p]);
        s_C1[pl[p]] = state[p] == 0 ? 0.f : (scale ? Tpre[p] * s.C1[p] : s.C1[p]);
        s_C2[pl[p]] = state[p] == 0 ? 0.f : (scale ? Tpre[p] * s.C2[p] : s.C2[p]);
        s_T[pl[p]] = scale ? Tpre[p] * s.T[p] : s.T[p];
        s_last[pl[p]] = state[p] == 0 ? 0u : s.last[p];
        s_state[pl[p]] = state[p];
    }
    cl.sync();
    // 4. CTA 0 adds the chunks in order and writes the pixels
    if (rank == 0) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            if (!inside[p]) continue;
            float C0 = 0.f, C1 = 0.f, C2 = 0.f, T = 1.f;
            unsigned last = 0;
            for (int j = 0; j < nc; ++j) {
                if (*cl.map_shared_rank(&s_state[pl[p]], j) == 0) continue;
                C0 += *cl.map_shared_rank(&s_C0[pl[p]], j);
                C1 += *cl.map_shared_rank(&s_C1[pl[p]], j);
                C2 += *cl.map_shared_rank(&s_C2[pl[p]], j);
                T = *cl.map_shared_rank(&s_T[pl[p]], j);
                const unsigned lj = *cl.map_shared_rank(&s_last[pl[p]], j);
                last = lj > 0 ? lj : last;
            }
            const long long pix = cam.pix0 + (long long)(tp.py0 + p) * cam.W + tp.px;
            rgba[pix] = make_float4(C0 + T * bg.x, C1 + T * bg.y, C2 + T * bg.z, 1.0f - T);
            final_T[pix] = T;
            last_out[pix] = last;
        }
    }
    cl.sync();  // the other CTAs' shared memory stays alive until CTA 0 has read it
}

// k_render over every tile whose run has at most split_min entries
static cudaError_t launch_render_tiles(const float2* xy, const float4* co, const float4* cd, long long n,
                                       const ivrgs_bins* b, const uint2* rg, const CamBatch& cb, float3 bgc,
                                       float4* out, float* final_T, uint32_t* last, int ppt, int sm, cudaStream_t s) {
    blend_shape(ppt, cb.th, [&](auto P, auto TH) {
        constexpr int kP = decltype(P)::value, kTH = decltype(TH)::value;
        k_render<kP, kTH><<<(unsigned)cb.n_tiles, kTile * kTH / kP, 0, s>>>(xy, co, cd, n, b->values, rg, cb, bgc, out,
                                                                          final_T, last, sm);
    });
    return cudaGetLastError();
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
    // with the split walk, runs longer than split_min go to the cluster kernel, on a side stream
    // beside k_render, which takes the rest; without it, k_render takes every tile
    const bool split = use_split(options().render_split, cb.n_tiles) && options().render_split != 3;
    const int sm = split ? options().render_split_min : INT_MAX;
    if (split && options().render_split == 4) {  // the long runs first, on the side stream, unsplit
        cudaStream_t side;
        cudaError_t e = split_fork(s, &side);
        if (e != cudaSuccess) return e;
        e = launch_render_tiles(xy, co, cd, p->n, b, rg, cb, bgc, out, final_T, last, ppt, -sm - 1, side);
        cudaError_t e2 = cudaSuccess;
        if (e == cudaSuccess) e2 = launch_render_tiles(xy, co, cd, p->n, b, rg, cb, bgc, out, final_T, last, ppt, sm, s);
        const cudaError_t e3 = split_join(s);
        return e != cudaSuccess ? e : (e2 != cudaSuccess ? e2 : e3);
    }
    if (split) {
        cudaStream_t side;
        cudaError_t e = split_fork(s, &side);
        if (e != cudaSuccess) return e;
        const unsigned grid = (unsigned)(cb.n_tiles * kSplit);
        blend_shape(ppt, cb.th, [&](auto P, auto TH) {
            constexpr int kP = decltype(P)::value, kTH = decltype(TH)::value;
            k_render_split<kP, kTH><<<grid, kTile * kTH / kP, 0, side>>>(xy, co, cd, p->n, b->values, rg, cb, bgc, sm,
                                                                       out, final_T, last);
        });
        e = cudaGetLastError();
        cudaError_t e2 = cudaSuccess;
        if (e == cudaSuccess) e2 = launch_render_tiles(xy, co, cd, p->n, b, rg, cb, bgc, out, final_T, last, ppt, sm, s);
        const cudaError_t e3 = split_join(s);
        return e != cudaSuccess ? e : (e2 != cudaSuccess ? e2 : e3);
    }
    return launch_render_tiles(xy, co, cd, p->n, b, rg, cb, bgc, out, final_T, last, ppt, sm, s);
}

}  // namespace ivrgs

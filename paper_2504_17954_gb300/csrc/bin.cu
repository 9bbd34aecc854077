// Tile binning and ordering (rows a3, a4 of the path).
//
// The result is the stable sort of all (tile, Gaussian) pairs by (global tile, float depth
// bits), ties in record order (view, Gaussian index). It is produced in two sorts instead of
// one sort of 64-bit keys over all pairs:
//
//   count:    per (view, Gaussian) record the number of covered tiles of its float32
//             rectangle (with IVRGS_BIN_CULL: of the rectangle's tiles that meet the
//             opacity cut-off ellipse, tile_cull.cuh), stored per record; per block of 2048
//             records the number of covered records and pairs;
//   compact:  the covered records, in record order, as (depth bits, compacted index), with
//             their pair counts and a packed 32-byte copy of what the emission needs;
//   sort 1:   stable LSD radix sort of the covered records by depth bits (4 onesweep passes);
//   count 2:  pair counts of the depth-ordered records (in that order), block and warp-range
//             sums, scan;
//   emit:     warp-cooperative emission of one (tile id, Gaussian) pair per covered tile, in
//             depth order, with the digit histograms of the tile ids: every warp takes its
//             own 256 records, 32 at a time; its lanes first stride over the row runs of the
//             32 records (one culling evaluation per run), then over the pairs of 32 runs at
//             a time, so stores stay coalesced (tile ids as u16 when they fit);
//   sort 2:   stable LSD radix sort of the pairs by tile id (one pass per 8 tile bits);
//   ranges:   [start, end) of every tile's run, written by the last pass of sort 2.
//
// Because sort 2 is stable and its input is in (depth, view, Gaussian) order, the output
// is ordered by (tile, depth, Gaussian) -- the same order as one stable sort by
// (tile << 32 | depth bits). Each onesweep pass ranks a tile of 4096 keys per CTA with warp
// ballots, publishes per-digit counts, orders the tile by digit in shared memory, resolves its
// global offsets by decoupled look-back over its predecessors (8 status words per round, a
// bounded spin), then scatters.
#include "common.cuh"
#include "tile_cull.cuh"

namespace ivrgs {

constexpr int kScanThreads = 256, kScanItems = 8, kScanBlock = kScanThreads * kScanItems;
constexpr int kSortThreads = 256, kSortItems = 16, kSortTile = kSortThreads * kSortItems;
constexpr int kMaxTilePasses = 4, kRecPasses = 4;
constexpr unsigned kFlagAgg = 1u << 30, kFlagPre = 2u << 30, kValMask = (1u << 30) - 1;
constexpr long long kMaxSpin = 1ll << 22;
constexpr int kLookWindow = 8;  // predecessors whose status words one look-back round reads

__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(unsigned* p, unsigned v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// view of record i = v * n + g (32-bit division whenever the records fit 32 bits)
__device__ __forceinline__ int view_of_record(long long i, long long n, long long total) {
    return total <= 0xffffffffll ? (int)((unsigned)i / (unsigned)n) : (int)(i / n);
}

// tile rows [ya, yb) of the rectangle whose band of pixel-centre rows [th ty + 0.5, th ty + th - 0.5]
// meets the ellipse's height [v - Y, v + Y] (the rows in it are still tested one by one)
__device__ __forceinline__ void cull_rows(const CullEll& e, int y0, int y1, int th, int& ya, int& yb) {
    ya = y0;
    yb = y1;
    if (e.mode == 2) return;
    if (e.mode == 0) {
        yb = ya;
        return;
    }
    const float inv = 1.0f / (float)th;  // exact: th is 16 or 8
    const float a = ceilf(__fmul_rn(__fsub_rn(__fsub_rn(e.v, e.Y), (float)th - 0.5f), inv));
    const float b = floorf(__fmul_rn(__fsub_rn(__fadd_rn(e.v, e.Y), 0.5f), inv)) + 1.0f;
    ya = (int)fminf(fmaxf(a, (float)y0), (float)y1);
    yb = (int)fminf(fmaxf(b, (float)ya), (float)y1);
}

// number of pairs of record i: every tile of its rectangle, or with culling the kept tiles
__device__ __forceinline__ unsigned record_pairs(float2 p, float4 co, int r, const CamDev& c, int th, int cull) {
    if (r <= 0) return 0u;
    int x0, x1, y0, y1;
    tile_rect(p.x, p.y, r, c.gx, c.gy, th, x0, x1, y0, y1);
    if (!(x1 > x0 && y1 > y0)) return 0u;
    if (!cull) return (unsigned)((x1 - x0) * (y1 - y0));
    const CullEll e = cull_setup(p, co, 1);
    int ya, yb;
    cull_rows(e, y0, y1, th, ya, yb);
    unsigned tot = 0;
    for (int ty = ya; ty < yb; ++ty) {
        int lo, hi;
        cull_row(e, ty, th, x0, x1, lo, hi);
        tot += (unsigned)(hi - lo);
    }
    return tot;
}

// block-wide exclusive scan of one u32 per thread (256 threads); returns the block total
__device__ __forceinline__ unsigned block_excl_scan(unsigned x, unsigned& excl, unsigned* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned w = lane < (kScanThreads / 32) ? s_warp[lane] : 0u;
        unsigned wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < (kScanThreads / 32)) s_warp[lane] = wi - w;
        if (lane == (kScanThreads / 32) - 1) s_warp[kScanThreads / 32] = wi;
    }
    __syncthreads();
    excl = s_warp[warp] + inc - x;
    const unsigned total = s_warp[kScanThreads / 32];
    __syncthreads();
    return total;
}

__device__ __forceinline__ unsigned warp_incl_scan(unsigned x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// number of items a sort/ranges kernel works on: the count, or 0 if it exceeds the buffer (an
// overflowing CAPACITY-mode call leaves the outputs unsorted; the caller sees the count)
__device__ __forceinline__ long long sort_count(const unsigned long long* d_n, long long cap) {
    const unsigned long long nn = *d_n;
    return (long long)nn <= cap ? (long long)nn : 0;
}

// ------------------------------------------------------------------------- count
// block sums: [0, nb) covered records, [nb, 2 nb) pairs; cnt[i] = pairs of record i
__global__ void __launch_bounds__(kScanThreads) k_count(const float2* __restrict__ xy,
                                                        const float4* __restrict__ conic_o,
                                                        const int* __restrict__ radius, long long n,
                                                        const __grid_constant__ CamBatch cb, int cull,
                                                        unsigned* __restrict__ cnt,
                                                        unsigned long long* __restrict__ sums, long long nb) {
    __shared__ unsigned s_red[2][kScanThreads / 32];
    const long long total = n * cb.n;
    const long long base = (long long)blockIdx.x * kScanBlock;
    unsigned vis = 0, pairs = 0;
    // the next record's loads are issued before this record's arithmetic (latency overlap)
    struct Rec {
        float2 p;
        float4 co;
        int r;
    };
    auto load = [&](long long i) {
        Rec q{};
        if (i < total) {
            q.r = radius[i];
            q.p = xy[i];
            q.co = conic_o[i];
        }
        return q;
    };
    Rec nxt = load(base + threadIdx.x);
#pragma unroll 1
    for (int j = 0; j < kScanItems; ++j) {
        const long long i = base + (long long)j * kScanThreads + threadIdx.x;
        const Rec q = nxt;
        if (j + 1 < kScanItems) nxt = load(i + kScanThreads);
        if (i < total) {
            const unsigned c = record_pairs(q.p, q.co, q.r, cb.c[view_of_record(i, n, total)], cb.th, cull);
            cnt[i] = c;
            vis += c ? 1u : 0u;
            pairs += c;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        vis += __shfl_xor_sync(0xffffffffu, vis, o);
        pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_red[0][threadIdx.x >> 5] = vis;
        s_red[1][threadIdx.x >> 5] = pairs;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long a = 0, b = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) {
            a += s_red[0][w];
            b += s_red[1][w];
        }
        sums[blockIdx.x] = a;
        sums[nb + blockIdx.x] = b;
    }
}

// ------------------------------------------------------------------------- scan of block sums
// exclusive scan of consecutive arrays of nb u64 (one CTA per array); array k's total goes to
// d_total0 (k = 0) or d_total1 (k = 1)
__global__ void __launch_bounds__(1024) k_scan_sums(unsigned long long* __restrict__ sums, long long nb,
                                                    unsigned long long* __restrict__ d_total0,
                                                    unsigned long long* __restrict__ d_total1) {
    __shared__ unsigned long long s_w[33];
    unsigned long long* a = sums + (long long)blockIdx.x * nb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long carry = 0;
    for (long long b0 = 0; b0 < nb; b0 += 1024) {
        const long long i = b0 + threadIdx.x;
        const unsigned long long x = i < nb ? a[i] : 0ull;
        unsigned long long inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_w[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = s_w[lane], wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            s_w[lane] = wi - w;
            if (lane == 31) s_w[32] = wi;
        }
        __syncthreads();
        if (i < nb) a[i] = carry + s_w[warp] + inc - x;
        carry += s_w[32];
        __syncthreads();
    }
    if (threadIdx.x == 0) *(blockIdx.x == 0 ? d_total0 : d_total1) = carry;
}

// ------------------------------------------------------------------------- compact
// Per covered record, in compacted order k: (depth bits, k) for the record sort, its pair count
// cnt2[k] and the packed record rec[2k..2k+1] = {(u, v, a, b), (c, o', record index, radius)}
// that the emission gathers in depth order (one 32-byte read instead of four scattered ones).
__global__ void __launch_bounds__(kScanThreads) k_compact(const unsigned* __restrict__ cnt,
                                                          const float2* __restrict__ xy,
                                                          const float4* __restrict__ conic_o,
                                                          const int* __restrict__ radius,
                                                          const float4* __restrict__ rgbd, long long total,
                                                          const unsigned long long* __restrict__ vis_off,
                                                          unsigned* __restrict__ rkey, unsigned* __restrict__ rval,
                                                          unsigned* __restrict__ cnt2, float4* __restrict__ rec,
                                                          unsigned* __restrict__ hist) {
    __shared__ unsigned s_hist[kRecPasses * 256];
    __shared__ unsigned s_warp[kScanThreads / 32 + 1];
    for (int k = threadIdx.x; k < kRecPasses * 256; k += kScanThreads) s_hist[k] = 0u;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kScanBlock;
    unsigned long long off = vis_off[blockIdx.x];
    // an item's loads are issued before the block scan that places it, and the next item's
    // before this item's stores, so that the scans overlap the memory latency
    struct Item {
        unsigned c, key;
        float2 p;
        float4 co;
        int r;
    };
    auto load = [&](long long i) {
        Item it{};
        if (i < total) {
            it.c = cnt[i];
            it.key = __float_as_uint(rgbd[i].w);
            it.p = xy[i];
            it.co = conic_o[i];
            it.r = radius[i];
        }
        return it;
    };
    Item nxt = load(base + threadIdx.x);
#pragma unroll 1
    for (int j = 0; j < kScanItems; ++j) {
        const long long i = base + (long long)j * kScanThreads + threadIdx.x;
        const Item it = nxt;
        if (j + 1 < kScanItems) nxt = load(i + kScanThreads);
        const unsigned c = it.c;
        const unsigned f = c ? 1u : 0u;
        unsigned excl;
        const unsigned tot = block_excl_scan(f, excl, s_warp);
        if (f) {
            const unsigned long long k = off + excl;
            const unsigned key = it.key;
            rkey[k] = key;
            rval[k] = (unsigned)k;
            cnt2[k] = c;
            rec[2 * k] = make_float4(it.p.x, it.p.y, it.co.x, it.co.y);
            rec[2 * k + 1] = make_float4(it.co.z, it.co.w, __uint_as_float((unsigned)i), __int_as_float(it.r));
#pragma unroll
            for (int q = 0; q < kRecPasses; ++q) atomicAdd(&s_hist[q * 256 + ((key >> (8 * q)) & 255u)], 1u);
        }
        off += tot;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kRecPasses * 256; k += kScanThreads)
        if (s_hist[k]) atomicAdd(&hist[k], s_hist[k]);
}

// ------------------------------------------------------------------------- count of sorted records
// pairs of the depth-ordered records: cnts[k] = pairs of the k-th record in depth order (so that
// the emission reads them in order), summed per block (sums[b], scanned afterwards) and per warp
// range (wsums[8 b + w]): warp w of block b covers the records [b kScanBlock + w kWarpRange,
// + kWarpRange), the unit the emission's warps work on
constexpr int kWarpRange = 32 * kScanItems;
constexpr int kScanWarps = kScanThreads / 32;
__global__ void __launch_bounds__(kScanThreads) k_count_sorted(const unsigned* __restrict__ cnt2,
                                                               const unsigned* __restrict__ rval,
                                                               const unsigned long long* __restrict__ d_m,
                                                               unsigned long long* __restrict__ sums,
                                                               unsigned* __restrict__ wsums,
                                                               unsigned* __restrict__ cnts) {
    __shared__ unsigned s_red[kScanWarps];
    const long long m = (long long)*d_m;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long base = (long long)blockIdx.x * kScanBlock + (long long)warp * kWarpRange;
    unsigned pairs = 0;
#pragma unroll 1
    for (int j = 0; j < kScanItems; ++j) {
        const long long k = base + j * 32 + lane;
        if (k < m) {
            const long long kk = rval[k];
            const unsigned c = kk < m ? cnt2[kk] : 0u;  // kk < m unless a timed-out sort left a slot unwritten
            cnts[k] = c;
            pairs += c;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
    if (lane == 0) {
        wsums[(long long)blockIdx.x * kScanWarps + warp] = pairs;
        s_red[warp] = pairs;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = 0;
        for (int w = 0; w < kScanWarps; ++w) b += s_red[w];
        sums[blockIdx.x] = b;
    }
}

// ------------------------------------------------------------------------- emission
// Every warp emits the pairs of its own range of kWarpRange depth-ordered records, 32 at a
// time, starting at the range's pair offset (no block-wide step, so a warp with large records
// does not hold up the others). First stage: its lanes stride over the 32 records' tile rows
// (row runs), evaluating each row's kept columns [lo, hi) once. Second stage, for every 32 row
// runs: its lanes stride over those runs' pairs, so consecutive lanes write consecutive slots.
// The pairs a warp writes must equal the sum of its records' counts from the count pass (the
// same rounded arithmetic decides both); a mismatch sets bit 1 of the error flag.
template <typename KT>
__global__ void __launch_bounds__(kScanThreads) k_emit(const float4* __restrict__ rec,
                                                       const unsigned* __restrict__ cnts, long long n,
                                                       const __grid_constant__ CamBatch cb, int cull,
                                                       const unsigned* __restrict__ rval,
                                                       const unsigned long long* __restrict__ d_m,
                                                       const unsigned long long* __restrict__ pair_off,
                                                       const unsigned* __restrict__ wsums,
                                                       KT* __restrict__ tiles, unsigned* __restrict__ vals,
                                                       long long cap, int n_passes, unsigned* __restrict__ hist,
                                                       unsigned* __restrict__ flag) {
    constexpr int kWarps = kScanThreads / 32;
    __shared__ unsigned s_hist[kMaxTilePasses * 256];
    __shared__ unsigned s_rti[kWarps][32];     // lane of the k-th of the warp's records with rows
    __shared__ unsigned s_rst[kWarps][32];     // its first row in the warp's row numbering
    __shared__ uint2 s_run[kWarps][32];        // k-th non-empty current run: (tile id - pair number, Gaussian)
    // per record of the current group, four 16-byte words (one vector load each per row):
    // (u, v, b/a, 1/a), (tau' a, det, Y, eyR), (mode, x0, x1, first row), (Gaussian, tile0, gx, -)
    __shared__ float4 s_ell0[kScanThreads], s_ell1[kScanThreads];
    __shared__ int4 s_rect[kScanThreads];
    __shared__ uint4 s_map[kScanThreads];
    for (int k = threadIdx.x; k < n_passes * 256; k += kScanThreads) s_hist[k] = 0u;
    __syncthreads();
    const long long m = (long long)*d_m;
    const long long total = n * cb.n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long base = (long long)blockIdx.x * kScanBlock + (long long)warp * kWarpRange;
    unsigned long long wbase = pair_off[blockIdx.x];  // + the pairs of the block's earlier warp ranges
    for (int w = 0; w < warp; ++w) wbase += wsums[(long long)blockIdx.x * kScanWarps + w];
#pragma unroll 1
    for (int j = 0; j < kScanItems; ++j) {
        const long long k = base + j * 32 + lane;
        if (__shfl_sync(0xffffffffu, k, 0) >= m) break;  // the rest of the range is past the end
        unsigned c = 0, rows = 0;
        {
            int x0 = 0, x1 = 0, y0 = 0, y1 = 0, ya = 0, yb = 0, v = 0;
            unsigned g = 0;
            CullEll e{};
            if (k < m) {
                const long long kk = rval[k];
                if (kk < m) {  // always true unless a timed-out sort left a slot unwritten
                    const float4 r0 = rec[2 * kk], r1 = rec[2 * kk + 1];
                    const long long i = __float_as_uint(r1.z);
                    const int r = __float_as_int(r1.w);
                    v = view_of_record(i, n, total);
                    g = (unsigned)(i - (long long)v * n);
                    c = cnts[k];
                    const float2 p = make_float2(r0.x, r0.y);
                    if (c && r > 0) {
                        tile_rect(p.x, p.y, r, cb.c[v].gx, cb.c[v].gy, cb.th, x0, x1, y0, y1);
                        e = cull_setup(p, make_float4(r0.z, r0.w, r1.x, r1.y), cull);
                        cull_rows(e, y0, y1, cb.th, ya, yb);
                        rows = (unsigned)(yb - ya);
                    }
                }
            }
            s_ell0[threadIdx.x] = make_float4(e.u, e.v, e.ba, e.inv_a);
            s_ell1[threadIdx.x] = make_float4(e.ta, e.det, e.Y, e.eyR);
            s_rect[threadIdx.x] = make_int4(e.mode, x0, x1, ya);
            s_map[threadIdx.x] = make_uint4(g, (unsigned)cb.c[v].tile0, (unsigned)cb.c[v].gx, 0u);
        }
        // records with rows, compacted: row rr belongs to the k-th of them, k = number of their
        // first rows at or before rr minus 1 (a 32-bit word of first rows per chunk of 32 rows)
        const unsigned rinc = warp_incl_scan(rows), rexcl = rinc - rows;
        const unsigned rnz = __ballot_sync(0xffffffffu, rows != 0u);
        if (rows) {
            const int k = __popc(rnz & ((1u << lane) - 1u));
            s_rti[warp][k] = (unsigned)lane;
            s_rst[warp][k] = rexcl;
        }
        const unsigned cwarp = __shfl_sync(0xffffffffu, warp_incl_scan(c), 31);
        __syncwarp();
        const unsigned R = __shfl_sync(0xffffffffu, rinc, 31);
        const unsigned upto = lane == 31 ? 0xffffffffu : (2u << lane) - 1u;  // positions <= lane
        unsigned done = 0, rcarry = 0;
        for (unsigned r0 = 0; r0 < R; r0 += 32) {
            const unsigned rr = r0 + lane;
            const unsigned rword = __reduce_or_sync(
                0xffffffffu, rows != 0u && rexcl >= r0 && rexcl - r0 < 32u ? 1u << (rexcl - r0) : 0u);
            int lo = 0, hi = 0;
            unsigned rowbase = 0, g = 0;
            if (rr < R) {
                const int k = (int)(rcarry + __popc(rword & upto)) - 1;
                const int ti = warp * 32 + (int)s_rti[warp][k];
                const float4 q0 = s_ell0[ti], q1 = s_ell1[ti];
                const int4 rc = s_rect[ti];
                const uint4 mp = s_map[ti];
                const CullEll e{q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, rc.x};
                const int ty = rc.w + (int)(rr - s_rst[warp][k]);
                cull_row(e, ty, cb.th, rc.y, rc.z, lo, hi);
                rowbase = mp.y + (unsigned)ty * mp.z;
                g = mp.x;
                if (hi > lo) {
                    // digits above the lowest byte: the run is contiguous in tile id (narrower
                    // than 256), so it adds to at most two digits per higher byte
                    const unsigned a = rowbase + (unsigned)lo, e = rowbase + (unsigned)hi;
                    for (int p = 1; p < n_passes; ++p) {
                        const unsigned sh = 8u * p, d0 = a >> sh, d1 = (e - 1u) >> sh;
                        if (d0 == d1) {
                            atomicAdd(&s_hist[p * 256 + (d0 & 255u)], e - a);
                        } else {
                            const unsigned B = d1 << sh;
                            atomicAdd(&s_hist[p * 256 + (d0 & 255u)], B - a);
                            atomicAdd(&s_hist[p * 256 + (d1 & 255u)], e - B);
                        }
                    }
                }
            }
            rcarry += __popc(rword);
            // the non-empty runs of these rows, compacted the same way over their pairs
            const unsigned w = (unsigned)(hi - lo);
            const unsigned pinc = warp_incl_scan(w), pexcl = pinc - w;
            const unsigned pnz = __ballot_sync(0xffffffffu, w != 0u);
            if (w) {
                const int k = __popc(pnz & ((1u << lane) - 1u));
                s_run[warp][k] = make_uint2(rowbase + (unsigned)lo - pexcl, g);  // tile of pair q = .x + q
            }
            __syncwarp();
            const unsigned W = __shfl_sync(0xffffffffu, pinc, 31);
            unsigned pcarry = 0;
            for (unsigned q0 = 0; q0 < W; q0 += 32) {
                const unsigned q = q0 + lane;
                const unsigned pword = __reduce_or_sync(
                    0xffffffffu, w != 0u && pexcl >= q0 && pexcl - q0 < 32u ? 1u << (pexcl - q0) : 0u);
                if (q < W) {
                    const int k = (int)(pcarry + __popc(pword & upto)) - 1;
                    const uint2 run = s_run[warp][k];
                    const unsigned tile = run.x + q;
                    const unsigned long long o = wbase + done + q;
                    if ((long long)o < cap) {
                        tiles[o] = (KT)tile;
                        vals[o] = run.y;
                        atomicAdd(&s_hist[tile & 255u], 1u);  // low byte: consecutive slots differ
                    }
                }
                pcarry += __popc(pword);
            }
            done += W;
            __syncwarp();
        }
        if (lane == 0 && done != cwarp) atomicOr(flag, 2u);
        wbase += cwarp;
        __syncwarp();
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n_passes * 256; k += kScanThreads)
        if (s_hist[k]) atomicAdd(&hist[k], s_hist[k]);
}

__global__ void k_hist_scan(const unsigned* __restrict__ hist, unsigned* __restrict__ base) {
    __shared__ unsigned s_warp[kScanThreads / 32 + 1];
    const unsigned x = hist[blockIdx.x * 256 + threadIdx.x];
    unsigned excl;
    block_excl_scan(x, excl, s_warp);
    base[blockIdx.x * 256 + threadIdx.x] = excl;
}

// ------------------------------------------------------------------------- onesweep pass
// LOOKBACK = true: onesweep (tiles taken in launch order from `counter`, offsets by decoupled
// look-back). LOOKBACK = false: the scatter of a reduce-then-scan pass (tile = block index,
// offsets read from `lookback`, which then holds the scanned digit table of k_upsweep and
// k_digit_scan: entry [d][tile] = first output slot of digit d in this tile).
// Keys are read as KIn and written as KOut (u32, or u16 for tile ids below 2^16 between the
// emission and the last pass, which writes u32); values are u32.
template <bool LOOKBACK, bool EARLY, typename KIn = unsigned, typename KOut = unsigned>
__global__ void __launch_bounds__(kSortThreads, 4) k_onesweep(const KIn* __restrict__ kin,
                                                           const unsigned* __restrict__ vin,
                                                           KOut* __restrict__ kout, unsigned* __restrict__ vout,
                                                           const unsigned long long* __restrict__ d_n, long long cap,
                                                           int shift, const unsigned* __restrict__ base,
                                                           unsigned* __restrict__ lookback,
                                                           unsigned* __restrict__ counter, unsigned* __restrict__ flag,
                                                           long long max_spin, long long skip_publish_tile,
                                                           int use_match, unsigned* __restrict__ ranges,
                                                           long long n_tiles) {
    __shared__ unsigned s_tile;
    __shared__ unsigned s_whist[kSortThreads / 32][256];
    __shared__ unsigned s_local[256];
    __shared__ unsigned s_global[256];
    __shared__ unsigned s_warp[kSortThreads / 32 + 1];
    __shared__ unsigned s_keys[kSortTile];
    __shared__ unsigned s_vals[kSortTile];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (LOOKBACK && tid == 0) s_tile = atomicAdd(counter, 1u);
    for (int k = tid; k < (kSortThreads / 32) * 256; k += kSortThreads) (&s_whist[0][0])[k] = 0u;
    __syncthreads();
    const long long tile = LOOKBACK ? (long long)s_tile : (long long)blockIdx.x;
    const long long n = sort_count(d_n, cap);
    const long long start = tile * kSortTile;
    if (start >= n) return;

    unsigned key[kSortItems], pos[kSortItems];
    const unsigned lt = (1u << lane) - 1u;
    // 32-bit offsets inside the radix tile; slots past the end hold the key 0xffffffff, whose
    // digit (255) ranks them after every real key of the tile (they are never written out)
    const int nvalid = (int)((n - start) < kSortTile ? (n - start) : kSortTile);
    const int wofs = warp * 32 * kSortItems + lane;
    const KIn* kin_t = kin + start;
    const unsigned* vin_t = vin + start;
    // values wait in shared memory, in input order, until their destinations are known
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const int li = wofs + j * 32;
        key[j] = li < nvalid ? (unsigned)kin_t[li] : 0xffffffffu;
        s_vals[li] = li < nvalid ? vin_t[li] : 0u;
    }
    const unsigned dg = (unsigned)tid;
    unsigned cnt = 0;
    if constexpr (EARLY) {
        // counts first: the tile's digit counts are published before the ranking, so that a
        // successor's look-back rarely finds this tile unpublished
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            // a bit-field extract of its own, so that the 16 digits are not kept live for the ranking
            unsigned dj;
            asm("bfe.u32 %0, %1, %2, 8;" : "=r"(dj) : "r"(key[j]), "r"(shift));
            const unsigned d0 = __shfl_sync(0xffffffffu, dj, 0);
            if (__all_sync(0xffffffffu, dj == d0)) {  // one digit across the warp: one update
                if (lane == 0) atomicAdd(&s_whist[warp][d0], 32u);
            } else {
                atomicAdd(&s_whist[warp][dj], 1u);
            }
        }
        __syncthreads();
        // per digit: warp-exclusive offsets (the ranking below continues from them)
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; ++w) {
            const unsigned c = s_whist[w][dg];
            s_whist[w][dg] = cnt;
            cnt += c;
        }
        if (LOOKBACK && tile != skip_publish_tile)
            st_relaxed(lookback + tile * 256 + dg, (tile == 0 ? kFlagPre : kFlagAgg) | cnt);
        unsigned lexcl;
        block_excl_scan(cnt, lexcl, s_warp);
        s_local[dg] = lexcl;
        s_global[dg] = cnt;  // parked until the look-back (not live across the ranking)
        __syncthreads();
    }
    // stable rank inside the warp, in (item, lane) order == index order
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const unsigned dj = (key[j] >> shift) & 255u;
        unsigned peers;
        if (use_match) {
            peers = __match_any_sync(0xffffffffu, dj);
        } else {
            peers = 0xffffffffu;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const unsigned bit = (dj >> b) & 1u;
                peers &= __ballot_sync(0xffffffffu, bit) ^ (bit - 1u);
            }
        }
        const unsigned before = s_whist[warp][dj];
        pos[j] = before + __popc(peers & lt);
        __syncwarp();
        if (lane == __ffs(peers) - 1) s_whist[warp][dj] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    if constexpr (!EARLY) {
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; ++w) {
            const unsigned c = s_whist[w][dg];
            s_whist[w][dg] = cnt;
            cnt += c;
        }
        if (LOOKBACK && tile != skip_publish_tile)
            st_relaxed(lookback + tile * 256 + dg, (tile == 0 ? kFlagPre : kFlagAgg) | cnt);
        unsigned lexcl;
        block_excl_scan(cnt, lexcl, s_warp);
        s_local[dg] = lexcl;
        __syncthreads();
    }
    // local scatter into digit order first, so that keys and ranks are dead during the look-back
    {
        unsigned val[kSortItems];
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const unsigned dj = (key[j] >> shift) & 255u;
            pos[j] += s_local[dj] + (EARLY ? 0u : s_whist[warp][dj]);
            s_keys[pos[j]] = key[j];
            val[j] = s_vals[wofs + j * 32];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) s_vals[pos[j]] = val[j];
    }
    if constexpr (!LOOKBACK) {
        s_global[dg] = lookback[(long long)dg * gridDim.x + tile];
    } else {
        // decoupled look-back: read the status words of up to kLookWindow predecessors at once, add
        // their counts nearest-first until one carries an inclusive prefix; wait (bounded) on a
        // predecessor that has not published yet
        unsigned prefix = 0;
        if (tile > 0) {
            long long t = tile - 1;  // nearest predecessor not yet accounted for
            long long spins = 0;
            bool done_lb = false;
            while (!done_lb) {
                unsigned st[kLookWindow];
    #pragma unroll
                for (int w = 0; w < kLookWindow; ++w)
                    st[w] = (t - w >= 0) ? ld_relaxed(lookback + (t - w) * 256 + dg) : (kFlagPre);
                int w = 0;
    #pragma unroll
                for (; w < kLookWindow; ++w) {
                    const unsigned f = st[w] >> 30;
                    if (f == 0u) break;  // not published yet: re-read from this tile
                    prefix += st[w] & kValMask;
                    if (f == 2u || t - w == 0) {
                        done_lb = true;
                        break;
                    }
                }
                if (done_lb) break;
                t -= w;
                if (w == 0) {
                    if (++spins > max_spin) {
                        atomicOr(flag, 1u);
                        break;
                    }
                    if (spins > 64) __nanosleep(64);
                }
            }
            if constexpr (EARLY) cnt = s_global[dg];
            if (tile != skip_publish_tile) st_relaxed(lookback + tile * 256 + dg, kFlagPre | ((prefix + cnt) & kValMask));
        }
        s_global[dg] = base[dg] + prefix;
    }
    __syncthreads();
    for (int i = tid; i < nvalid; i += kSortThreads) {
        const unsigned k = s_keys[i];
        const unsigned dd = (k >> shift) & 255u;
        const unsigned o = s_global[dd] + ((unsigned)i - s_local[dd]);
        kout[o] = (KOut)k;
        vout[o] = s_vals[i];
        if (ranges != nullptr) {
            // last pass: the tile is fully ordered by key, so equal keys form runs, and where a run
            // begins the previous one ends. Inside a digit's stretch of this tile both boundaries are
            // final (plain stores). At the first item of a digit an earlier tile may hold more of
            // either key, so the start of this key and the end of the previous one are candidates:
            // atomic maxima of ~start and of end against the zeroed table (k_ranges_fix decodes)
            const unsigned kp = i > 0 ? s_keys[i - 1] : 0xffffffffu;
            if (kp != k) {
                const unsigned dp = (kp >> shift) & 255u;
                const bool inner = i > 0 && dp == dd;
                if ((long long)k < n_tiles) {
                    if (inner) ranges[2ll * k] = ~o;
                    else atomicMax(&ranges[2ll * k], ~o);
                }
                if (i > 0 && (long long)kp < n_tiles) {
                    if (inner) ranges[2ll * kp + 1] = o;
                    else atomicMax(&ranges[2ll * kp + 1], s_global[dp] + ((unsigned)i - s_local[dp]));
                }
            }
            if (i == nvalid - 1 && (long long)k < n_tiles) atomicMax(&ranges[2ll * k + 1], o + 1u);
        }
    }
}

// ranges written by the last radix pass: start stored complemented; an untouched tile is empty
__global__ void __launch_bounds__(256) k_ranges_fix(unsigned* __restrict__ ranges, long long n_tiles) {
    const long long t = (long long)blockIdx.x * 256 + threadIdx.x;
    if (t >= n_tiles) return;
    uint2 r = reinterpret_cast<uint2*>(ranges)[t];
    if (r.y == 0u) {
        r.x = 0u;
    } else {
        r.x = ~r.x;
        if (r.x > r.y) r.x = r.y;  // only after a timed-out sort (reported); keeps the run empty
    }
    reinterpret_cast<uint2*>(ranges)[t] = r;
}

// ------------------------------------------------------------------------- reduce-then-scan
// k_upsweep: digit histogram of radix tile blockIdx.x, written to table[d][tile] (zeros for a
// tile past the end). k_digit_scan: one CTA per digit d turns row d into exclusive offsets
// base[d] + sum of the row's earlier tiles.
__global__ void __launch_bounds__(kSortThreads) k_upsweep(const unsigned* __restrict__ kin,
                                                          const unsigned long long* __restrict__ d_n, long long cap,
                                                          int shift, unsigned* __restrict__ table) {
    __shared__ unsigned s_h[256];
    const int tid = threadIdx.x;
    s_h[tid] = 0u;
    __syncthreads();
    const long long n = sort_count(d_n, cap);
    const long long start = (long long)blockIdx.x * kSortTile;
    if (start < n) {
        const int nvalid = (int)((n - start) < kSortTile ? (n - start) : kSortTile);
        const unsigned* k = kin + start;
#pragma unroll 4
        for (int j = tid; j < nvalid; j += kSortThreads) atomicAdd(&s_h[(k[j] >> shift) & 255u], 1u);
    }
    __syncthreads();
    table[(long long)tid * gridDim.x + blockIdx.x] = s_h[tid];
}

constexpr int kDigitScanThreads = 1024, kDigitScanItems = 16;

__global__ void __launch_bounds__(kDigitScanThreads) k_digit_scan(unsigned* __restrict__ table,
                                                                  const unsigned* __restrict__ base, long long n_tiles) {
    __shared__ unsigned s_w[kDigitScanThreads / 32 + 1];
    unsigned* row = table + (long long)blockIdx.x * n_tiles;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned carry = base[blockIdx.x];
    for (long long c0 = 0; c0 < n_tiles; c0 += (long long)kDigitScanThreads * kDigitScanItems) {
        const long long t0 = c0 + (long long)threadIdx.x * kDigitScanItems;
        unsigned v[kDigitScanItems], sum = 0;
#pragma unroll
        for (int k = 0; k < kDigitScanItems; ++k) {
            v[k] = t0 + k < n_tiles ? row[t0 + k] : 0u;
            sum += v[k];
        }
        unsigned inc = warp_incl_scan(sum);
        if (lane == 31) s_w[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const unsigned w = s_w[lane];
            const unsigned wi = warp_incl_scan(w);
            s_w[lane] = wi - w;
            if (lane == 31) s_w[32] = wi;
        }
        __syncthreads();
        unsigned run = carry + s_w[warp] + inc - sum;
#pragma unroll
        for (int k = 0; k < kDigitScanItems; ++k)
            if (t0 + k < n_tiles) {
                row[t0 + k] = run;
                run += v[k];
            }
        carry += s_w[32];
        __syncthreads();
    }
}

// ------------------------------------------------------------------------- ranges
// from the sorted tile ids (the single-tile case, which has no radix pass to write them)
__global__ void __launch_bounds__(256) k_ranges(const unsigned* __restrict__ tiles,
                                                const unsigned long long* __restrict__ d_n, long long cap,
                                                long long n_tiles, unsigned* __restrict__ ranges) {
    const long long n = sort_count(d_n, cap);
    const long long i0 = ((long long)blockIdx.x * 256 + threadIdx.x) * 4;  // four consecutive pairs
    if (i0 >= n) return;
    unsigned t[4];
    if (i0 + 4 <= n) {
        const uint4 q = *reinterpret_cast<const uint4*>(tiles + i0);  // 16-byte aligned: i0 % 4 == 0
        t[0] = q.x; t[1] = q.y; t[2] = q.z; t[3] = q.w;
    } else {
        for (int k = 0; k < 4; ++k) t[k] = i0 + k < n ? tiles[i0 + k] : 0xffffffffu;
    }
    unsigned prev = i0 > 0 ? tiles[i0 - 1] : 0xffffffffu;
    const unsigned next = i0 + 4 < n ? tiles[i0 + 4] : 0xffffffffu;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const long long i = i0 + k;
        if (i >= n) break;
        const unsigned tk = t[k];
        const unsigned nx = k < 3 ? t[k + 1] : next;
        if ((long long)tk < n_tiles) {  // always, unless a timed-out sort left a slot unwritten
            if (i == 0 || prev != tk) ranges[2ll * tk] = (unsigned)i;
            if (i == n - 1 || nx != tk) ranges[2ll * tk + 1] = (unsigned)(i + 1);
        }
        prev = tk;
    }
}

// ------------------------------------------------------------------------- host side
static size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

BinPlan plan_bin(long long n_records, long long n_tiles, long long capacity) {
    BinPlan p{};
    int tile_bits = 0;
    while (tile_bits < 32 && (1ll << tile_bits) < n_tiles) ++tile_bits;
    p.key_bits = tile_bits;
    p.n_passes = (tile_bits + 7) / 8;
    p.n_records = n_records;
    p.n_scan_blocks = (n_records + kScanBlock - 1) / kScanBlock;
    p.capacity = capacity;
    p.rec_tiles = (n_records + kSortTile - 1) / kSortTile;
    p.sort_tiles = (capacity + kSortTile - 1) / kSortTile;
    const size_t nb = (size_t)(p.n_scan_blocks > 0 ? p.n_scan_blocks : 1);
    const size_t nr = (size_t)(n_records > 0 ? n_records : 1);
    const size_t cp = (size_t)(capacity > 0 ? capacity : 1);
    // [flag | histograms | digit bases | pass counters | totals] are cleared by every call;
    // the error flag stays at offset 0 so that ivrgs_bin_check can find it without the plan
    size_t o = 0;
    p.off_flag = o;         o = align_up(o + 4);
    p.off_hist = o;         o = align_up(o + 4 * 256 * (kRecPasses + kMaxTilePasses));
    p.off_base = o;         o = align_up(o + 4 * 256 * (kRecPasses + kMaxTilePasses));
    p.off_counter = o;      o = align_up(o + 4 * (kRecPasses + kMaxTilePasses));
    p.off_total = o;        o = align_up(o + 8 * 2);
    p.clear_bytes = o;
    p.off_block_sums = o;   o = align_up(o + 8 * 3 * nb + 4 * (kScanThreads / 32) * nb);
    p.off_rec = o;          o = align_up(o + 4 * 4 * nr);
    p.off_cnt = o;          o = align_up(o + 4 * nr);
    p.off_cnt2 = o;         o = align_up(o + 4 * nr);
    p.off_prec = o;         o = align_up(o + 32 * nr);
    p.off_lookback_rec = o; o = align_up(o + 4 * 256 * (size_t)kRecPasses * (size_t)(p.rec_tiles > 0 ? p.rec_tiles : 1));
    p.off_lookback = o;     o = align_up(o + 4 * 256 * (size_t)(p.n_passes > 0 ? p.n_passes : 1) *
                                         (size_t)(p.sort_tiles > 0 ? p.sort_tiles : 1));
    p.off_keys_alt = o;     o = align_up(o + 4 * cp);
    p.off_vals_alt = o;     o = align_up(o + 4 * cp);
    p.total_bytes = o;
    return p;
}

// the debug hook used by the failure-detection test: a look-back bound and a radix tile that
// skips publishing (host-side injection; every wait stays bounded)
static long long g_max_spin = kMaxSpin;
static long long g_skip_publish_tile = -1;

struct BinBufs {
    unsigned long long *sums, *d_m, *d_n;
    unsigned *hist_rec, *hist_tile, *base_rec, *base_tile, *counter, *flag, *lb_rec, *lb_tile;
    unsigned *rkey[2], *rval[2], *talt, *valt, *cnt, *cnt2;
    float4* prec;
};

static BinBufs bufs(const BinPlan& plan, char* ws, ivrgs_bins* out) {
    BinBufs b;
    const size_t nr = (size_t)(plan.n_records > 0 ? plan.n_records : 1);
    b.sums = reinterpret_cast<unsigned long long*>(ws + plan.off_block_sums);
    b.hist_rec = reinterpret_cast<unsigned*>(ws + plan.off_hist);
    b.hist_tile = b.hist_rec + 256 * kRecPasses;
    b.base_rec = reinterpret_cast<unsigned*>(ws + plan.off_base);
    b.base_tile = b.base_rec + 256 * kRecPasses;
    b.counter = reinterpret_cast<unsigned*>(ws + plan.off_counter);
    b.flag = reinterpret_cast<unsigned*>(ws + plan.off_flag);
    b.d_m = reinterpret_cast<unsigned long long*>(ws + plan.off_total);
    b.d_n = reinterpret_cast<unsigned long long*>(out->d_n_pairs);
    unsigned* r = reinterpret_cast<unsigned*>(ws + plan.off_rec);
    b.rkey[0] = r; b.rval[0] = r + nr; b.rkey[1] = r + 2 * nr; b.rval[1] = r + 3 * nr;
    b.lb_rec = reinterpret_cast<unsigned*>(ws + plan.off_lookback_rec);
    b.lb_tile = reinterpret_cast<unsigned*>(ws + plan.off_lookback);
    b.talt = reinterpret_cast<unsigned*>(ws + plan.off_keys_alt);
    b.valt = reinterpret_cast<unsigned*>(ws + plan.off_vals_alt);
    b.cnt = reinterpret_cast<unsigned*>(ws + plan.off_cnt);
    b.cnt2 = reinterpret_cast<unsigned*>(ws + plan.off_cnt2);
    b.prec = reinterpret_cast<float4*>(ws + plan.off_prec);
    return b;
}

cudaError_t launch_bin_count(const ivrgs_projected* p, const CamBatch& cb, const BinPlan& plan, int cull, char* ws,
                             uint64_t* d_n_pairs, cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(ws, 0, plan.clear_bytes, s)) != cudaSuccess) return e;
    unsigned long long* sums = reinterpret_cast<unsigned long long*>(ws + plan.off_block_sums);
    unsigned long long* d_m = reinterpret_cast<unsigned long long*>(ws + plan.off_total);
    const long long nb = plan.n_scan_blocks;
    if (nb > 0) {
        IVRGS_PROF("k_count", s);
        k_count<<<(unsigned)nb, kScanThreads, 0, s>>>(reinterpret_cast<const float2*>(p->xy),
                                                      reinterpret_cast<const float4*>(p->conic_o), p->radius, p->n,
                                                      cb, cull, reinterpret_cast<unsigned*>(ws + plan.off_cnt), sums,
                                                      nb);
    }
    {
        IVRGS_PROF("k_scan_sums", s);
        k_scan_sums<<<2, 1024, 0, s>>>(sums, nb, d_m, reinterpret_cast<unsigned long long*>(d_n_pairs));
    }
    return cudaGetLastError();
}

// key16: the keys between passes are u16 (the first pass reads u16, the last writes u32)
static cudaError_t onesweep_passes(int n_passes, void* k0, unsigned* v0, void* k1, unsigned* v1,
                                   const unsigned long long* d_n, long long cap, const unsigned* base,
                                   unsigned* lookback, long long tiles, unsigned* counter, unsigned* flag,
                                   bool early, bool key16, unsigned* ranges, long long n_tiles, const char* name,
                                   cudaStream_t s) {
    void* kb[2] = {k0, k1};
    unsigned* vb[2] = {v0, v1};
    const bool rts = options().sort_scan != 0;
    using u16 = unsigned short;
    for (int ps = 0; ps < n_passes && tiles > 0; ++ps) {
        const int src = ps & 1, dst = src ^ 1;
        unsigned* lb = lookback + (size_t)256 * ps * tiles;
        unsigned* rg = ps == n_passes - 1 ? ranges : nullptr;
        const unsigned* bs = base + 256 * ps;
        const long long ms = g_max_spin, skip = g_skip_publish_tile;
        const int mt = options().sort_match;
        IVRGS_PROF(name, s);
        if (rts) {
            k_upsweep<<<(unsigned)tiles, kSortThreads, 0, s>>>(static_cast<const unsigned*>(kb[src]), d_n, cap, 8 * ps, lb);
            k_digit_scan<<<256, kDigitScanThreads, 0, s>>>(lb, bs, tiles);
            k_onesweep<false, false><<<(unsigned)tiles, kSortThreads, 0, s>>>(
                static_cast<const unsigned*>(kb[src]), vb[src], static_cast<unsigned*>(kb[dst]), vb[dst], d_n, cap,
                8 * ps, bs, lb, counter + ps, flag, ms, skip, mt, rg, n_tiles);
        } else if (early) {
            k_onesweep<true, true><<<(unsigned)tiles, kSortThreads, 0, s>>>(
                static_cast<const unsigned*>(kb[src]), vb[src], static_cast<unsigned*>(kb[dst]), vb[dst], d_n, cap,
                8 * ps, bs, lb, counter + ps, flag, ms, skip, mt, rg, n_tiles);
        } else if (key16 && ps < n_passes - 1) {
            k_onesweep<true, false, u16, u16><<<(unsigned)tiles, kSortThreads, 0, s>>>(
                static_cast<const u16*>(kb[src]), vb[src], static_cast<u16*>(kb[dst]), vb[dst], d_n, cap, 8 * ps, bs,
                lb, counter + ps, flag, ms, skip, mt, rg, n_tiles);
        } else if (key16) {
            k_onesweep<true, false, u16, unsigned><<<(unsigned)tiles, kSortThreads, 0, s>>>(
                static_cast<const u16*>(kb[src]), vb[src], static_cast<unsigned*>(kb[dst]), vb[dst], d_n, cap, 8 * ps,
                bs, lb, counter + ps, flag, ms, skip, mt, rg, n_tiles);
        } else {
            k_onesweep<true, false><<<(unsigned)tiles, kSortThreads, 0, s>>>(
                static_cast<const unsigned*>(kb[src]), vb[src], static_cast<unsigned*>(kb[dst]), vb[dst], d_n, cap,
                8 * ps, bs, lb, counter + ps, flag, ms, skip, mt, rg, n_tiles);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_bin_sort(const ivrgs_projected* p, const CamBatch& cb, const BinPlan& plan, int cull, char* ws,
                            ivrgs_bins* out, long long exact_pairs, cudaStream_t s) {
    cudaError_t e;
    BinBufs b = bufs(plan, ws, out);
    const long long cap = out->capacity;
    const long long nb = plan.n_scan_blocks;
    const long long rec_tiles = plan.rec_tiles;
    const long long n_work = exact_pairs >= 0 ? (exact_pairs < cap ? exact_pairs : cap) : cap;
    const long long pair_tiles = (n_work + kSortTile - 1) / kSortTile;
    if (rec_tiles > 0 &&
        (e = cudaMemsetAsync(b.lb_rec, 0, 4 * 256 * (size_t)kRecPasses * (size_t)rec_tiles, s)) != cudaSuccess)
        return e;
    if (pair_tiles > 0 && plan.n_passes > 0 &&
        (e = cudaMemsetAsync(b.lb_tile, 0, 4 * 256 * (size_t)plan.n_passes * (size_t)pair_tiles, s)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(out->ranges, 0, 8 * (size_t)out->n_tiles, s)) != cudaSuccess) return e;
    const float2* xy = reinterpret_cast<const float2*>(p->xy);
    // covered records in record order, then by depth
    if (nb > 0) {
        IVRGS_PROF("k_compact", s);
        k_compact<<<(unsigned)nb, kScanThreads, 0, s>>>(b.cnt, xy, reinterpret_cast<const float4*>(p->conic_o),
                                                        p->radius, reinterpret_cast<const float4*>(p->rgbd),
                                                        plan.n_records, b.sums, b.rkey[0], b.rval[0], b.cnt2, b.prec,
                                                        b.hist_rec);
    }
    {
        IVRGS_PROF("k_hist_scan", s);
        k_hist_scan<<<kRecPasses, 256, 0, s>>>(b.hist_rec, b.base_rec);
    }
    if ((e = onesweep_passes(kRecPasses, b.rkey[0], b.rval[0], b.rkey[1], b.rval[1], b.d_m, plan.n_records,
                             b.base_rec, b.lb_rec, rec_tiles, b.counter, b.flag, true, false, nullptr, 0, "k_onesweep_rec",
                             s)) != cudaSuccess)
        return e;
    // pair offsets of the depth-ordered records
    unsigned long long* sums2 = b.sums + 2 * (nb > 0 ? nb : 1);
    unsigned* wsums = reinterpret_cast<unsigned*>(sums2 + (nb > 0 ? nb : 1));
    if (nb > 0) {
        IVRGS_PROF("k_count_sorted", s);
        // (the record-order counts are dead after the compaction: their buffer takes the sorted ones)
        k_count_sorted<<<(unsigned)nb, kScanThreads, 0, s>>>(b.cnt2, b.rval[0], b.d_m, sums2, wsums, b.cnt);
    }
    {
        IVRGS_PROF("k_scan_sums", s);
        k_scan_sums<<<1, 1024, 0, s>>>(sums2, nb, b.d_n, b.d_n);
    }
    // pairs in depth order, then stable by tile; the last pass lands in the caller's arrays
    // tile ids below 2^16 travel as u16 between the emission and the last pass (6 bytes per pair
    // instead of 8 through every pass but the last), in the default pass form
    const bool key16 = plan.n_passes >= 1 && plan.key_bits <= 16 && options().sort_scan == 0 &&
                       options().sort_early == 0;
    unsigned *t0, *v0, *t1, *v1;
    if (plan.n_passes % 2 == 0) {
        t0 = out->tiles; v0 = out->values; t1 = b.talt; v1 = b.valt;
    } else {
        t0 = b.talt; v0 = b.valt; t1 = out->tiles; v1 = out->values;
    }
    if (nb > 0) {
        IVRGS_PROF("k_emit", s);
        if (key16)
            k_emit<unsigned short><<<(unsigned)nb, kScanThreads, 0, s>>>(
                b.prec, b.cnt, p->n, cb, cull, b.rval[0], b.d_m, sums2, wsums, reinterpret_cast<unsigned short*>(t0),
                v0, cap, plan.n_passes, b.hist_tile, b.flag);
        else
            k_emit<unsigned><<<(unsigned)nb, kScanThreads, 0, s>>>(b.prec, b.cnt, p->n, cb, cull, b.rval[0], b.d_m,
                                                                  sums2, wsums, t0, v0, cap, plan.n_passes,
                                                                  b.hist_tile, b.flag);
    }
    if (plan.n_passes > 0) {
        IVRGS_PROF("k_hist_scan", s);
        k_hist_scan<<<plan.n_passes, 256, 0, s>>>(b.hist_tile, b.base_tile);
    }
    if ((e = onesweep_passes(plan.n_passes, t0, v0, t1, v1, b.d_n, cap, b.base_tile, b.lb_tile, pair_tiles,
                             b.counter + kRecPasses, b.flag, options().sort_early != 0, key16, out->ranges,
                             out->n_tiles, "k_onesweep", s)) != cudaSuccess)
        return e;
    if (plan.n_passes > 0 && pair_tiles > 0) {  // the last pass wrote the runs
        IVRGS_PROF("k_ranges_fix", s);
        k_ranges_fix<<<(unsigned)((out->n_tiles + 255) / 256), 256, 0, s>>>(out->ranges, out->n_tiles);
    } else if (n_work > 0) {  // a single tile: no radix pass
        IVRGS_PROF("k_ranges", s);
        k_ranges<<<(unsigned)((n_work + 1023) / 1024), 256, 0, s>>>(out->tiles, b.d_n, cap, out->n_tiles,
                                                                   out->ranges);
    }
    return cudaGetLastError();
}

}  // namespace ivrgs

extern "C" void ivrgs_debug_bin_hooks(long long max_spin, long long skip_publish_tile) {
    ivrgs::g_max_spin = max_spin > 0 ? max_spin : ivrgs::kMaxSpin;
    ivrgs::g_skip_publish_tile = skip_publish_tile;
}

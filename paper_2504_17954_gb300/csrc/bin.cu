// Tile binning and the (tile, depth) key sort (rows a3, a4 of the path).
//
//   count:  per (view, Gaussian) record the number of covered tiles of its float32 rectangle,
//           summed per block of 2048 records;
//   scan:   exclusive scan of the block sums (one CTA) and the total pair count;
//   emit:   block-level scan of the record counts in record order, one (key, value) pair per
//           covered tile, and the 8-bit digit histograms of all sort passes;
//   sort:   stable LSD radix sort, one onesweep kernel per 8-bit digit: each CTA ranks a tile
//           of 3072 keys with warp match/popc, publishes its per-digit counts and resolves its
//           per-digit offsets by decoupled look-back over its predecessors (bounded spin),
//           then scatters through shared memory;
//   ranges: [start, end) of each tile's run in the sorted keys.
#include "common.cuh"

namespace ivrgs {

constexpr int kScanThreads = 256, kScanItems = 8, kScanBlock = kScanThreads * kScanItems;
constexpr int kSortThreads = 256, kSortItems = 12, kSortTile = kSortThreads * kSortItems;
constexpr int kMaxPasses = 8;
constexpr unsigned kFlagAgg = 1u << 30, kFlagPre = 2u << 30, kValMask = (1u << 30) - 1;
constexpr long long kMaxSpin = 1ll << 22;

__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(unsigned* p, unsigned v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned record_count(const float2* __restrict__ xy, const int* __restrict__ radius,
                                                 long long i, const CamDev& c, int& x0, int& x1, int& y0, int& y1) {
    const int r = radius[i];
    if (r <= 0) return 0u;
    const float2 p = xy[i];
    tile_rect(p.x, p.y, r, c.gx, c.gy, x0, x1, y0, y1);
    return (unsigned)((x1 - x0) * (y1 - y0));
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

// ------------------------------------------------------------------------- count
__global__ void __launch_bounds__(kScanThreads) k_count(const float2* __restrict__ xy, const int* __restrict__ radius,
                                                        long long n, const __grid_constant__ CamBatch cb,
                                                        unsigned long long* __restrict__ block_sums) {
    __shared__ unsigned s_red[kScanThreads / 32];
    const long long total = n * cb.n;
    const long long base = (long long)blockIdx.x * kScanBlock;
    unsigned long long sum = 0;
    int x0, x1, y0, y1;
#pragma unroll 1
    for (int j = 0; j < kScanItems; ++j) {
        const long long i = base + (long long)j * kScanThreads + threadIdx.x;
        if (i < total) sum += record_count(xy, radius, i, cb.c[i / n], x0, x1, y0, y1);
    }
    unsigned s = (unsigned)sum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) b += s_red[w];
        block_sums[blockIdx.x] = b;
    }
}

// ------------------------------------------------------------------------- scan of block sums
__global__ void __launch_bounds__(1024) k_scan_sums(unsigned long long* __restrict__ sums, long long nb,
                                                    unsigned long long* __restrict__ d_total) {
    __shared__ unsigned long long s_w[33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long carry = 0;
    for (long long b0 = 0; b0 < nb; b0 += 1024) {
        const long long i = b0 + threadIdx.x;
        const unsigned long long x = i < nb ? sums[i] : 0ull;
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
        if (i < nb) sums[i] = carry + s_w[warp] + inc - x;
        carry += s_w[32];
        __syncthreads();
    }
    if (threadIdx.x == 0) *d_total = carry;
}

// ------------------------------------------------------------------------- emit + histograms
__global__ void __launch_bounds__(kScanThreads) k_emit(const float2* __restrict__ xy, const int* __restrict__ radius,
                                                       const float4* __restrict__ rgbd, long long n,
                                                       const __grid_constant__ CamBatch cb,
                                                       const unsigned long long* __restrict__ block_off,
                                                       unsigned long long* __restrict__ keys,
                                                       unsigned* __restrict__ vals, long long cap, int n_passes,
                                                       unsigned* __restrict__ hist) {
    __shared__ unsigned s_hist[kMaxPasses * 256];
    __shared__ unsigned s_warp[kScanThreads / 32 + 1];
    for (int k = threadIdx.x; k < n_passes * 256; k += kScanThreads) s_hist[k] = 0u;
    __syncthreads();
    const long long total = n * cb.n;
    const long long base = (long long)blockIdx.x * kScanBlock;
    unsigned long long off = block_off[blockIdx.x];
#pragma unroll 1
    for (int j = 0; j < kScanItems; ++j) {
        const long long i = base + (long long)j * kScanThreads + threadIdx.x;
        int x0 = 0, x1 = 0, y0 = 0, y1 = 0, v = 0;
        unsigned c = 0;
        if (i < total) {
            v = (int)(i / n);
            c = record_count(xy, radius, i, cb.c[v], x0, x1, y0, y1);
        }
        unsigned excl;
        const unsigned tot = block_excl_scan(c, excl, s_warp);
        if (c) {
            const CamDev& cam = cb.c[v];
            const unsigned dbits = __float_as_uint(rgbd[i].w);
            const unsigned g = (unsigned)(i - (long long)v * n);
            unsigned long long o = off + excl;
            for (int ty = y0; ty < y1; ++ty)
                for (int tx = x0; tx < x1; ++tx, ++o) {
                    const unsigned long long tile = (unsigned long long)(cam.tile0 + (long long)ty * cam.gx + tx);
                    const unsigned long long key = (tile << 32) | dbits;
                    if ((long long)o < cap) {
                        keys[o] = key;
                        vals[o] = g;
                        for (int p = 0; p < n_passes; ++p) atomicAdd(&s_hist[p * 256 + ((key >> (8 * p)) & 255)], 1u);
                    }
                }
        }
        off += tot;
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
__global__ void __launch_bounds__(kSortThreads) k_onesweep(const unsigned long long* __restrict__ kin,
                                                           const unsigned* __restrict__ vin,
                                                           unsigned long long* __restrict__ kout,
                                                           unsigned* __restrict__ vout,
                                                           const unsigned long long* __restrict__ d_n, long long cap,
                                                           int shift, const unsigned* __restrict__ base,
                                                           unsigned* __restrict__ lookback,
                                                           unsigned* __restrict__ counter, unsigned* __restrict__ flag,
                                                           long long max_spin, long long skip_publish_tile) {
    __shared__ unsigned s_tile;
    __shared__ unsigned s_whist[kSortThreads / 32][256];
    __shared__ unsigned s_local[256];
    __shared__ unsigned s_global[256];
    __shared__ unsigned s_warp[kSortThreads / 32 + 1];
    __shared__ unsigned long long s_keys[kSortTile];
    __shared__ unsigned s_vals[kSortTile];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(counter, 1u);
    for (int k = tid; k < (kSortThreads / 32) * 256; k += kSortThreads) (&s_whist[0][0])[k] = 0u;
    __syncthreads();
    const long long tile = s_tile;
    const unsigned long long nn = *d_n;
    const long long n = (long long)nn < cap ? (long long)nn : cap;
    const long long start = tile * kSortTile;
    if (start >= n) return;

    unsigned long long k[kSortItems];
    unsigned d[kSortItems], pos[kSortItems];
    const unsigned lt = (1u << lane) - 1u;
    const long long wbase = start + (long long)warp * 32 * kSortItems;
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const long long idx = wbase + j * 32 + lane;
        const bool valid = idx < n;
        k[j] = valid ? kin[idx] : 0ull;
        d[j] = valid ? (unsigned)((k[j] >> shift) & 255u) : 256u;
    }
    // rank inside the warp, in (item, lane) order == index order
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const unsigned peers = __match_any_sync(0xffffffffu, d[j]);
        const unsigned before = d[j] < 256u ? s_whist[warp][d[j]] : 0u;
        pos[j] = before + __popc(peers & lt);
        __syncwarp();
        if (d[j] < 256u && lane == __ffs(peers) - 1) s_whist[warp][d[j]] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit (thread = digit): prefix over warps and the tile's count
    const unsigned dg = (unsigned)tid;
    unsigned cnt = 0;
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; ++w) {
        const unsigned c = s_whist[w][dg];
        s_whist[w][dg] = cnt;
        cnt += c;
    }
    unsigned* my_status = lookback + tile * 256 + dg;
    const bool publish = tile != skip_publish_tile;
    if (publish) st_relaxed(my_status, (tile == 0 ? kFlagPre : kFlagAgg) | cnt);
    unsigned lexcl;
    block_excl_scan(cnt, lexcl, s_warp);
    s_local[dg] = lexcl;
    // decoupled look-back
    unsigned prefix = 0;
    if (tile > 0) {
        long long t = tile - 1;
        long long spins = 0;
        while (true) {
            const unsigned s = ld_relaxed(lookback + t * 256 + dg);
            const unsigned f = s >> 30;
            if (f == 0u) {
                if (++spins > max_spin) {
                    atomicOr(flag, 1u);
                    break;
                }
                if (spins > 64) __nanosleep(64);
                continue;
            }
            prefix += s & kValMask;
            if (f == 2u || t == 0) break;
            --t;
        }
        if (publish) st_relaxed(my_status, kFlagPre | ((prefix + cnt) & kValMask));
    }
    s_global[dg] = base[dg] + prefix;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kSortItems; ++j)
        if (d[j] < 256u) {
            pos[j] += s_local[d[j]] + s_whist[warp][d[j]];
            s_keys[pos[j]] = k[j];
        }
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const long long idx = wbase + j * 32 + lane;
        if (d[j] < 256u) s_vals[pos[j]] = vin[idx];
    }
    __syncthreads();
    const int nvalid = (int)((n - start) < kSortTile ? (n - start) : kSortTile);
    for (int i = tid; i < nvalid; i += kSortThreads) {
        const unsigned long long key = s_keys[i];
        const unsigned dd = (unsigned)((key >> shift) & 255u);
        const unsigned o = s_global[dd] + ((unsigned)i - s_local[dd]);
        kout[o] = key;
        vout[o] = s_vals[i];
    }
}

// ------------------------------------------------------------------------- ranges
__global__ void k_ranges(const unsigned long long* __restrict__ keys, const unsigned long long* __restrict__ d_n,
                         long long cap, unsigned* __restrict__ ranges) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long nn = *d_n;
    const long long n = (long long)nn < cap ? (long long)nn : cap;
    if (i >= n) return;
    const unsigned long long t = keys[i] >> 32;
    if (i == 0 || (keys[i - 1] >> 32) != t) ranges[2 * t] = (unsigned)i;
    if (i == n - 1 || (keys[i + 1] >> 32) != t) ranges[2 * t + 1] = (unsigned)(i + 1);
}

// ------------------------------------------------------------------------- host side
static size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

BinPlan plan_bin(long long n_records, long long n_tiles, long long capacity) {
    BinPlan p{};
    int tile_bits = 0;
    while (tile_bits < 32 && (1ll << tile_bits) < n_tiles) ++tile_bits;
    p.key_bits = 32 + tile_bits;
    p.n_passes = (p.key_bits + 7) / 8;
    p.n_records = n_records;
    p.n_scan_blocks = (n_records + kScanBlock - 1) / kScanBlock;
    p.capacity = capacity;
    p.sort_tiles = (capacity + kSortTile - 1) / kSortTile;
    // [flag | histograms | digit bases | pass counters | total] are cleared by every sort;
    // the error flag stays at offset 0 so that ivrgs_bin_check can find it without the plan
    size_t o = 0;
    p.off_flag = o;       o = align_up(o + 4);
    p.off_hist = o;       o = align_up(o + 4 * kMaxPasses * 256);
    p.off_base = o;       o = align_up(o + 4 * kMaxPasses * 256);
    p.off_counter = o;    o = align_up(o + 4 * kMaxPasses);
    p.off_total = o;      o = align_up(o + 8);
    p.off_block_sums = o; o = align_up(o + 8 * (size_t)(p.n_scan_blocks > 0 ? p.n_scan_blocks : 1));
    p.off_lookback = o;   o = align_up(o + 4 * 256 * (size_t)p.n_passes * (size_t)(p.sort_tiles > 0 ? p.sort_tiles : 1));
    p.off_keys_alt = o;   o = align_up(o + 8 * (size_t)(capacity > 0 ? capacity : 1));
    p.off_vals_alt = o;   o = align_up(o + 4 * (size_t)(capacity > 0 ? capacity : 1));
    p.total_bytes = o;
    return p;
}

// the debug hook used by the failure-detection test: a look-back bound and a tile that skips
// publishing (host-side injection; every wait stays bounded)
static long long g_max_spin = kMaxSpin;
static long long g_skip_publish_tile = -1;

cudaError_t launch_bin_count(const ivrgs_projected* p, const CamBatch& cb, const BinPlan& plan, char* ws,
                             uint64_t* d_n_pairs, cudaStream_t s) {
    unsigned long long* sums = reinterpret_cast<unsigned long long*>(ws + plan.off_block_sums);
    if (plan.n_scan_blocks > 0) {
        IVRGS_PROF("k_count", s);
        k_count<<<(unsigned)plan.n_scan_blocks, kScanThreads, 0, s>>>(
            reinterpret_cast<const float2*>(p->xy), p->radius, p->n, cb, sums);
    }
    {
        IVRGS_PROF("k_scan_sums", s);
        k_scan_sums<<<1, 1024, 0, s>>>(sums, plan.n_scan_blocks, reinterpret_cast<unsigned long long*>(d_n_pairs));
    }
    return cudaGetLastError();
}

cudaError_t launch_bin_sort(const ivrgs_projected* p, const CamBatch& cb, const BinPlan& plan, char* ws,
                            ivrgs_bins* out, long long exact_pairs, cudaStream_t s) {
    cudaError_t e;
    unsigned long long* sums = reinterpret_cast<unsigned long long*>(ws + plan.off_block_sums);
    unsigned* hist = reinterpret_cast<unsigned*>(ws + plan.off_hist);
    unsigned* base = reinterpret_cast<unsigned*>(ws + plan.off_base);
    unsigned* counter = reinterpret_cast<unsigned*>(ws + plan.off_counter);
    unsigned* flag = reinterpret_cast<unsigned*>(ws + plan.off_flag);
    unsigned* lookback = reinterpret_cast<unsigned*>(ws + plan.off_lookback);
    unsigned long long* kalt = reinterpret_cast<unsigned long long*>(ws + plan.off_keys_alt);
    unsigned* valt = reinterpret_cast<unsigned*>(ws + plan.off_vals_alt);
    const unsigned long long* d_n = reinterpret_cast<const unsigned long long*>(out->d_n_pairs);
    const long long cap = out->capacity;
    unsigned long long* out_keys = reinterpret_cast<unsigned long long*>(out->keys);
    // tiles actually launched per pass: exact count when known, else the capacity bound
    const long long n_work = exact_pairs >= 0 ? (exact_pairs < cap ? exact_pairs : cap) : cap;
    const long long sort_tiles = (n_work + kSortTile - 1) / kSortTile;
    // clear histograms, counters, flag (contiguous) and the look-back words of the launched tiles
    if ((e = cudaMemsetAsync(ws, 0, plan.off_block_sums, s)) != cudaSuccess) return e;
    if (sort_tiles > 0 &&
        (e = cudaMemsetAsync(lookback, 0, 4 * 256 * (size_t)plan.n_passes * (size_t)sort_tiles, s)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(out->ranges, 0, 8 * (size_t)out->n_tiles, s)) != cudaSuccess) return e;
    // ping-pong so that the last pass lands in the caller's arrays
    unsigned long long* kb[2];
    unsigned* vb[2];
    if (plan.n_passes % 2 == 0) {
        kb[0] = out_keys; vb[0] = out->values; kb[1] = kalt; vb[1] = valt;
    } else {
        kb[0] = kalt; vb[0] = valt; kb[1] = out_keys; vb[1] = out->values;
    }
    if (plan.n_scan_blocks > 0) {
        IVRGS_PROF("k_emit", s);
        k_emit<<<(unsigned)plan.n_scan_blocks, kScanThreads, 0, s>>>(
            reinterpret_cast<const float2*>(p->xy), p->radius, reinterpret_cast<const float4*>(p->rgbd), p->n, cb,
            sums, kb[0], vb[0], cap, plan.n_passes, hist);
    }
    {
        IVRGS_PROF("k_hist_scan", s);
        k_hist_scan<<<plan.n_passes, 256, 0, s>>>(hist, base);
    }
    for (int ps = 0; ps < plan.n_passes && sort_tiles > 0; ++ps) {
        const int src = ps & 1, dst = src ^ 1;
        {
            IVRGS_PROF("k_onesweep", s);
            k_onesweep<<<(unsigned)sort_tiles, kSortThreads, 0, s>>>(
                kb[src], vb[src], kb[dst], vb[dst], d_n, cap, 8 * ps, base + 256 * ps,
                lookback + (size_t)256 * ps * sort_tiles, counter + ps, flag, g_max_spin, g_skip_publish_tile);
        }
    }
    if (n_work > 0) {
        IVRGS_PROF("k_ranges", s);
        k_ranges<<<(unsigned)((n_work + 255) / 256), 256, 0, s>>>(out_keys, d_n, cap, out->ranges);
    }
    return cudaGetLastError();
}

}  // namespace ivrgs

extern "C" void ivrgs_debug_bin_hooks(long long max_spin, long long skip_publish_tile) {
    ivrgs::g_max_spin = max_spin > 0 ? max_spin : ivrgs::kMaxSpin;
    ivrgs::g_skip_publish_tile = skip_publish_tile;
}

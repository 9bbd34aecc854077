// Shared device-side definitions of libivrgs (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "ivrgs.h"
#include "prof.cuh"

namespace ivrgs {

constexpr int kTile = 16;              // tile width (pixels); the tile height is 16 or 8 (CamBatch::th)
constexpr float kGuard = 1.3f;         // guard band of x/z, y/z inside the Jacobian
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;
constexpr float kLog2e = 1.4426950408889634f;

// Camera as the kernels see it (travels in kernel parameter space).
struct CamDev {
    int W, H, gx, gy;
    long long tile0, pix0;
    float fx, fy, cx, cy;
    float R[9], t[3], campos[3];
    float znear, limx, limy;
    int headlight;
    float light[3];   // normalised light_dir (orbital light)
    float light_len;  // |light_dir|
};

struct CamBatch {
    int n;
    int th;  // tile height (pixels): 16 or 8; tiles are kTile wide
    long long n_tiles;
    CamDev c[IVRGS_MAX_VIEWS];
};

// view of a global tile id (binary search over the per-view first tile)
__device__ __forceinline__ int view_of_tile(const CamBatch& cb, long long t) {
    int lo = 0, hi = cb.n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (cb.c[mid].tile0 <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// float32 tile rectangle, half-open: x0 = clamp(floor((u - r)/kTile), 0, G), x1 = clamp(floor((u + r)/kTile)
// + 1, 0, G), and the same in y with the tile height th
__device__ __forceinline__ void tile_rect(float u, float v, int r, int gx, int gy, int th, int& x0, int& x1,
                                          int& y0, int& y1) {
    const float fr = (float)r;
    const float inv = 1.0f / (float)kTile;  // exact: power of two
    const float invh = 1.0f / (float)th;    // exact: th is 16 or 8
    float a = floorf(__fmul_rn(__fsub_rn(u, fr), inv));
    float b = floorf(__fmul_rn(__fadd_rn(u, fr), inv)) + 1.0f;
    float c = floorf(__fmul_rn(__fsub_rn(v, fr), invh));
    float d = floorf(__fmul_rn(__fadd_rn(v, fr), invh)) + 1.0f;
    x0 = (int)fminf(fmaxf(a, 0.0f), (float)gx);
    x1 = (int)fminf(fmaxf(b, 0.0f), (float)gx);
    y0 = (int)fminf(fmaxf(c, 0.0f), (float)gy);
    y1 = (int)fminf(fmaxf(d, 0.0f), (float)gy);
}

__device__ __forceinline__ float fast_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---------------------------------------------------------------------------------------
// host-side helpers
// ---------------------------------------------------------------------------------------
void set_error(const std::string& msg);
ivrgs_status cuda_status(cudaError_t e, const char* what);

struct BinPlan {
    int n_passes;          // 8-bit digit passes of the tile-id sort
    int key_bits;          // bits of the tile ids
    long long n_records;   // n * n_views
    long long n_scan_blocks;
    long long capacity;
    long long rec_tiles;   // radix tiles of the record sort
    long long sort_tiles;  // radix tiles of the pair sort at full capacity
    // workspace layout (byte offsets); [0, clear_bytes) is zeroed by every call
    size_t off_flag, off_hist, off_base, off_counter, off_total, clear_bytes, off_block_sums, off_rec,
        off_cnt, off_cnt2, off_prec, off_lookback_rec, off_lookback, off_keys_alt, off_vals_alt, total_bytes;
};

// tile heights the kernels are built for
inline bool tile_height_ok(int th) { return th == 16 || th == 8; }
ivrgs_status make_cam_batch(const ivrgs_camera* cams, int32_t n_views, CamBatch* cb, int th = kTile);

// tunable launch shapes (set through ivrgs_set_option; read by the launchers)
struct Options {
    int render_ppt = 0;      // pixels per thread of the forward blend (1, 2, 4 or 8; 0 = by tile count)
    int render_bwd_ppt = 0;  // pixels per thread of the backward blend (1, 2, 4 or 8; 0 = by tile count)
    int sort_match = 0;      // radix ranking: 0 = warp ballots per digit bit, 1 = match.any
    int sort_scan = 0;       // radix offsets: 0 = decoupled look-back (onesweep), 1 = reduce-then-scan
    int sort_early = 0;      // radix tile: 1 = publish its digit counts before ranking (look-back waits less)
    int render_split = 0;    // blends: 0 = split long runs over a CTA cluster when the call has fewer
                             // than kSplitTiles tiles (the default), 1 = always, 2 = never, 3 = the
                             // backward only (by tile count), 4 = no split, but the long runs in a
                             // launch of their own, first (by tile count)
    int render_split_min = 256;  // entries per chunk at least (a run this long or shorter is one chunk)
};
Options& options();
// Pixels per thread of a blend launch over n_tiles tiles: the option, or with 0 (the default) a
// choice by occupancy. Four pixels per thread (64-thread CTAs, 18 per SM: ~2,700 at a time on
// 152 SMs) issue the fewest instructions per pixel and win once the tiles fill the GPU more than
// once (measured on GB300: 4,096 and 26,000 tiles); below that each CTA's walk is latency-bound
// and more warps per tile (fewer pixels per thread) finish sooner (64 and 2,500 tiles): one pixel
// per thread in both blends, where each warp also walks only the entries that reach its two rows
// (the single 800^2 view: 1.254 ms per step against 1.313 with the forward at two).
constexpr long long kAutoPptTiles = 3072;
inline int blend_ppt(int option, long long n_tiles, bool backward) {
    (void)backward;
    if (option != 0) return option;
    return n_tiles >= kAutoPptTiles ? 4 : 1;
}
// Split walk (a cluster of CTAs per tile, each compositing a chunk of the run) for a blend launch
// over n_tiles tiles: the option, or by default below two tiles per SM, where the heaviest tiles'
// serial walks are the launch (measured on GB300: the 10k-Gaussian 128^2 view, 64 tiles, 2.5x
// faster fwd+bwd; the 800^2 view, 2500 tiles, 0.7x: there the split's extra work outweighs it).
constexpr long long kSplitTiles = 304;
inline bool use_split(int option, long long n_tiles) {
    if (option == 1) return true;
    if (option == 2) return false;
    return n_tiles < kSplitTiles;  // 0, 3 and 4 (the forward checks for 3 itself)
}
BinPlan plan_bin(long long n_records, long long n_tiles, long long capacity);

// Fork/join of the split walk: the cluster kernel of the long runs runs on a library stream
// beside the caller's stream's kernel of the other tiles. fork() makes the side stream wait for
// the caller's stream and returns it; join() makes the caller's stream wait for the side
// stream. One side stream and two events per device, created on first use and kept for the
// process; fork() holds a lock until join() so that host threads cannot interleave the pair.
// Both steps are capturable (the side stream joins an ongoing capture of the caller's stream).
cudaError_t split_fork(cudaStream_t s, cudaStream_t* side);
cudaError_t split_join(cudaStream_t s);

// launchers (each returns cudaGetLastError() of its launches)
cudaError_t launch_compose(const ivrgs_gaussians* models, int32_t n_models, ivrgs_gaussians* composed,
                           cudaStream_t s);
cudaError_t launch_edit_table(const ivrgs_model_edit* edits, int32_t n_models, const ivrgs_light* light,
                              float* table, cudaStream_t s);
cudaError_t launch_morton(const ivrgs_gaussians* g, const float* lo, const float* hi, uint64_t* keys, cudaStream_t s);
cudaError_t launch_pack_mixed(const ivrgs_gaussians* in, const uint32_t* order, ivrgs_gaussians* out,
                              cudaStream_t s);
cudaError_t launch_project(const ivrgs_gaussians* g, const float* table, const CamBatch& cb, float lowpass,
                           ivrgs_projected* out, cudaStream_t s);
cudaError_t launch_bin_count(const ivrgs_projected* p, const CamBatch& cb, const BinPlan& plan, int cull, char* ws,
                             uint64_t* d_n_pairs, cudaStream_t s);
cudaError_t launch_bin_sort(const ivrgs_projected* p, const CamBatch& cb, const BinPlan& plan, int cull, char* ws,
                            ivrgs_bins* out, long long exact_pairs, cudaStream_t s);
cudaError_t launch_render(const ivrgs_projected* p, const ivrgs_bins* b, const CamBatch& cb, const float* bg,
                          float* rgba, float* final_T, uint32_t* last, cudaStream_t s);
cudaError_t launch_render_aux(const ivrgs_gaussians* g, const float* table, const ivrgs_projected* p,
                              const ivrgs_bins* b, const CamBatch& cb, float* aux, cudaStream_t s);
size_t vq_workspace(int n_models, int K);
cudaError_t launch_vq_build(const ivrgs_gaussians* g, int K, int iters, ivrgs_gaussians* out, char* ws,
                            cudaStream_t s);
size_t image_loss_workspace(const CamBatch& cb, long long n_pix);
cudaError_t launch_image_loss(const float* rgba, const float* target, const CamBatch& cb, long long n_pix,
                              float lambda, char* ws, float* loss, float* dL, cudaStream_t s);
cudaError_t launch_edit_adam_init(const float* table, int n_models, float* state, cudaStream_t s);
cudaError_t launch_edit_adam(float* table, const float* egrad, int n_models, float* state, int flags, float lr,
                             float b1, float b2, float eps, cudaStream_t s);
cudaError_t launch_render_backward(const ivrgs_gaussians* g, const float* table, const ivrgs_projected* p,
                                   const ivrgs_bins* b, const CamBatch& cb, float lowpass, const float* bg,
                                   const float* final_T, const uint32_t* last, const float* dL, char* ws,
                                   ivrgs_gaussians* grad, float* edit_grad, int accumulate, cudaStream_t s);
// the projection's reverse mode from the per-(view, Gaussian) gradients of the 2D quantities
// g0 (du, dv, da, db), g1 (dc, do', dr, dg), g2 (db) (the second half of the backward)
cudaError_t launch_project_backward(const ivrgs_gaussians* g, const float* table, const CamBatch& cb, float lowpass,
                                    const float4* g0, const float4* g1, const float* g2, ivrgs_gaussians* grad,
                                    float* edit_grad, int accumulate, cudaStream_t s);
size_t aux_backward_workspace(long long n, int n_views);
cudaError_t launch_render_aux_backward(const ivrgs_gaussians* g, const float* table, const ivrgs_projected* p,
                                       const ivrgs_bins* b, const CamBatch& cb, float lowpass, const float* final_T,
                                       const uint32_t* last, const float* dL, char* ws, ivrgs_gaussians* grad,
                                       float* edit_grad, cudaStream_t s);

}  // namespace ivrgs

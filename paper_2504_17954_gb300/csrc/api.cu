// Host entry points of libivrgs: argument checks, camera packing, launches.
#include <math.h>

#include <cstdio>
#include <algorithm>
#include <mutex>
#include <string>

#include "common.cuh"

namespace ivrgs {

static thread_local std::string g_last_error;

Options& options() {
    static Options o;
    return o;
}

void set_error(const std::string& msg) { g_last_error = msg; }

namespace {
struct SideStream {
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
constexpr int kMaxSideDevices = 64;
SideStream g_side[kMaxSideDevices];
std::mutex g_side_mu;       // guards creation
std::mutex g_side_pair_mu;  // held from split_fork to split_join
int g_side_dev = -1;
}  // namespace

cudaError_t split_fork(cudaStream_t s, cudaStream_t* side) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxSideDevices) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lk(g_side_mu);
        SideStream& ss = g_side[dev];
        if (!ss.side) {
            if ((e = cudaStreamCreateWithFlags(&ss.side, cudaStreamNonBlocking)) != cudaSuccess) return e;
            if ((e = cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming)) != cudaSuccess) return e;
            if ((e = cudaEventCreateWithFlags(&ss.join, cudaEventDisableTiming)) != cudaSuccess) return e;
        }
    }
    g_side_pair_mu.lock();
    g_side_dev = dev;
    SideStream& ss = g_side[dev];
    if ((e = cudaEventRecord(ss.fork, s)) != cudaSuccess || (e = cudaStreamWaitEvent(ss.side, ss.fork, 0)) != cudaSuccess) {
        g_side_pair_mu.unlock();
        return e;
    }
    *side = ss.side;
    return cudaSuccess;
}

cudaError_t split_join(cudaStream_t s) {
    SideStream& ss = g_side[g_side_dev];
    cudaError_t e = cudaEventRecord(ss.join, ss.side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ss.join, 0);
    g_side_pair_mu.unlock();
    return e;
}

ivrgs_status cuda_status(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return IVRGS_OK;
    set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return IVRGS_ERR_CUDA;
}

static ivrgs_status invalid(const std::string& msg) {
    set_error(msg);
    return IVRGS_ERR_INVALID_ARG;
}

static bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

ivrgs_status make_cam_batch(const ivrgs_camera* cams, int32_t n_views, CamBatch* cb, int th) {
    if (!tile_height_ok(th)) {
        set_error("tiles are 16 pixels wide and 16 or 8 high (got height " + std::to_string(th) + ")");
        return IVRGS_ERR_UNSUPPORTED;
    }
    if (!cams) return invalid("cams is NULL");
    if (n_views < 1 || n_views > IVRGS_MAX_VIEWS)
        return invalid("n_views must be in [1, " + std::to_string(IVRGS_MAX_VIEWS) + "]");
    cb->n = n_views;
    cb->th = th;
    long long tiles = 0;
    for (int v = 0; v < n_views; ++v) {
        const ivrgs_camera& c = cams[v];
        if (c.W <= 0 || c.H <= 0 || c.W > 32768 || c.H > 32768)
            return invalid("camera " + std::to_string(v) + ": W and H must be in [1, 32768]");
        if (!(c.fx > 0.f) || !(c.fy > 0.f) || !isfinite(c.fx) || !isfinite(c.fy))
            return invalid("camera " + std::to_string(v) + ": focal lengths must be positive and finite");
        if (c.pix_offset < 0) return invalid("camera " + std::to_string(v) + ": negative pix_offset");
        CamDev& d = cb->c[v];
        d.W = c.W;
        d.H = c.H;
        d.gx = (c.W + kTile - 1) / kTile;
        d.gy = (c.H + th - 1) / th;
        d.tile0 = tiles;
        tiles += (long long)d.gx * d.gy;
        d.pix0 = c.pix_offset;
        d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
        for (int k = 0; k < 9; ++k) d.R[k] = c.R[k];
        for (int k = 0; k < 3; ++k) { d.t[k] = c.t[k]; d.campos[k] = c.campos[k]; }
        d.znear = c.znear;
        d.limx = kGuard * (0.5f * (float)c.W) / c.fx;
        d.limy = kGuard * (0.5f * (float)c.H) / c.fy;
        d.headlight = c.headlight ? 1 : 0;
        const float ll = sqrtf(c.light_dir[0] * c.light_dir[0] + c.light_dir[1] * c.light_dir[1] +
                               c.light_dir[2] * c.light_dir[2]);
        if (!c.headlight && !(ll > 0.f)) return invalid("camera " + std::to_string(v) + ": zero light_dir");
        d.light_len = ll > 0.f ? ll : 1.f;
        for (int k = 0; k < 3; ++k) d.light[k] = ll > 0.f ? c.light_dir[k] / ll : 0.f;
    }
    // views must not overlap in the packed image
    for (int v = 0; v < n_views; ++v)
        for (int u = v + 1; u < n_views; ++u) {
            const long long a0 = cams[v].pix_offset, a1 = a0 + (long long)cams[v].W * cams[v].H;
            const long long b0 = cams[u].pix_offset, b1 = b0 + (long long)cams[u].W * cams[u].H;
            if (a0 < b1 && b0 < a1)
                return invalid("cameras " + std::to_string(v) + " and " + std::to_string(u) + " overlap in pix_offset");
        }
    cb->n_tiles = tiles;
    return IVRGS_OK;
}

static ivrgs_status check_gaussians(const ivrgs_gaussians* g, const char* name, bool need_model_id,
                                    bool allow_mixed = false) {
    if (!g) return invalid(std::string(name) + " is NULL");
    if (g->n < 0) return invalid(std::string(name) + ": negative n");
    if (g->precision != IVRGS_FP32 && g->precision != IVRGS_MIXED && g->precision != IVRGS_VQ)
        return invalid(std::string(name) + ": unknown precision");
    if (g->precision != IVRGS_FP32 && !allow_mixed) {
        set_error(std::string(name) + ": this call takes IVRGS_FP32 storage");
        return IVRGS_ERR_UNSUPPORTED;
    }
    if (g->n == 0) return IVRGS_OK;
    if (!g->mean || !g->log_scale || !g->quat || !g->opacity_logit || !g->dcolor || !g->normal || !g->kads ||
        (need_model_id && !g->model_id))
        return invalid(std::string(name) + ": NULL attribute array");
    if (g->precision == IVRGS_FP32) {
        if (!aligned(g->quat, 16) || !aligned(g->kads, 16))
            return invalid(std::string(name) + ": quat and kads must be 16-byte aligned");
        if (!aligned(g->mean, 4) || !aligned(g->log_scale, 4) || !aligned(g->dcolor, 4) || !aligned(g->normal, 4) ||
            !aligned(g->opacity_logit, 4))
            return invalid(std::string(name) + ": misaligned attribute array");
    } else if (g->precision == IVRGS_VQ) {
        if (!g->codebook) return invalid(std::string(name) + ": IVRGS_VQ needs the codebook array");
        if (g->vq_k < 1 || g->vq_k > IVRGS_VQ_MAX_K) return invalid(std::string(name) + ": vq_k out of range");
        if (!aligned(g->quat, 4) || !aligned(g->kads, 4) || !aligned(g->mean, 4) || !aligned(g->normal, 4) ||
            !aligned(g->codebook, 4))
            return invalid(std::string(name) + ": IVRGS_VQ quat/kads indices must be 4-byte aligned");
        if (!g->model_id) return invalid(std::string(name) + ": IVRGS_VQ needs model_id");
    } else {
        if (!g->anchor) return invalid(std::string(name) + ": IVRGS_MIXED needs the anchor array");
        if (!aligned(g->quat, 8) || !aligned(g->kads, 8))
            return invalid(std::string(name) + ": IVRGS_MIXED quat and kads must be 8-byte aligned");
        if (!aligned(g->mean, 2) || !aligned(g->log_scale, 2) || !aligned(g->dcolor, 2) || !aligned(g->normal, 2) ||
            !aligned(g->opacity_logit, 2) || !aligned(g->anchor, 4))
            return invalid(std::string(name) + ": misaligned attribute array");
    }
    if (need_model_id && !aligned(g->model_id, 2)) return invalid(std::string(name) + ": misaligned model_id");
    if (g->sh) {
        if (g->sh_degree < 0 || g->sh_degree > 3) return invalid(std::string(name) + ": sh_degree must be 0..3");
        if (!aligned(g->sh, 4)) return invalid(std::string(name) + ": misaligned sh");
    }
    return IVRGS_OK;
}

static ivrgs_status check_projected(const ivrgs_projected* p, int64_t n, int32_t n_views) {
    if (!p) return invalid("projected is NULL");
    if (p->n != n || p->n_views != n_views) return invalid("projected: n / n_views do not match");
    if (n == 0) return IVRGS_OK;
    if (!p->xy || !p->conic_o || !p->rgbd || !p->radius) return invalid("projected: NULL array");
    if (!aligned(p->xy, 8) || !aligned(p->conic_o, 16) || !aligned(p->rgbd, 16) || !aligned(p->radius, 4))
        return invalid("projected: misaligned array (xy 8, conic_o/rgbd 16 bytes)");
    return IVRGS_OK;
}

static ivrgs_status check_bins(const ivrgs_bins* b, const CamBatch& cb) {
    if (!b) return invalid("bins is NULL");
    if (b->tile_w != kTile || !tile_height_ok(b->tile_h)) {
        set_error("bins: tiles are 16 pixels wide and 16 or 8 high");
        return IVRGS_ERR_UNSUPPORTED;
    }
    if (b->tile_h != cb.th) return invalid("bins: tile_h does not match the camera batch");
    if (b->n_tiles != cb.n_tiles)
        return invalid("bins: n_tiles = " + std::to_string(b->n_tiles) + " but the cameras have " +
                       std::to_string(cb.n_tiles) + " tiles");
    if (b->capacity < 0 || b->capacity >= IVRGS_MAX_PAIRS) return invalid("bins: capacity must be in [0, 2^30)");
    if (!b->ranges || !b->d_n_pairs || (b->capacity > 0 && (!b->tiles || !b->values)))
        return invalid("bins: NULL array");
    if (!aligned(b->tiles, 4) || !aligned(b->values, 4) || !aligned(b->ranges, 8) || !aligned(b->d_n_pairs, 8))
        return invalid("bins: misaligned array (tiles/values 4, ranges/d_n_pairs 8 bytes)");
    return IVRGS_OK;
}

}  // namespace ivrgs

using namespace ivrgs;

extern "C" {

const char* ivrgs_last_error(void) { return g_last_error.c_str(); }

int32_t ivrgs_version(void) { return 100; }

ivrgs_status ivrgs_set_option(const char* name, int64_t value) {
    set_error("");
    if (!name) return invalid("name is NULL");
    const std::string k(name);
    if (k == "render_pixels_per_thread" || k == "render_bwd_pixels_per_thread") {
        if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8)
            return invalid(k + " must be 0 (by tile count), 1, 2, 4 or 8");
        (k == "render_pixels_per_thread" ? options().render_ppt : options().render_bwd_ppt) = (int)value;
        return IVRGS_OK;
    }
    if (k == "render_split") {
        if (value < 0 || value > 4)
            return invalid(k + " must be 0 (by tile count), 1 (always), 2 (never), 3 (backward only) or 4 (long "
                               "runs first, unsplit)");
        options().render_split = (int)value;
        return IVRGS_OK;
    }
    if (k == "render_split_min") {
        bool ok = false;
        for (int c : {32, 64, 128, 256, 384, 512, 768, 1024, 2048, 4096}) ok = ok || value == c;
        if (!ok) return invalid(k + " must be one of 32, 64, 128, 256, 384, 512, 768, 1024, 2048, 4096");
        options().render_split_min = (int)value;
        return IVRGS_OK;
    }
    if (k == "sort_match" || k == "sort_scan" || k == "sort_early") {
        if (value != 0 && value != 1) return invalid(k + " must be 0 or 1");
        (k == "sort_match" ? options().sort_match : k == "sort_scan" ? options().sort_scan : options().sort_early) =
            (int)value;
        return IVRGS_OK;
    }
    return invalid("unknown option '" + k + "'");
}

ivrgs_status ivrgs_get_option(const char* name, int64_t* value) {
    set_error("");
    if (!name || !value) return invalid("NULL argument");
    const std::string k(name);
    if (k == "render_pixels_per_thread") *value = options().render_ppt;
    else if (k == "render_bwd_pixels_per_thread") *value = options().render_bwd_ppt;
    else if (k == "sort_match") *value = options().sort_match;
    else if (k == "sort_scan") *value = options().sort_scan;
    else if (k == "sort_early") *value = options().sort_early;
    else if (k == "render_split") *value = options().render_split;
    else if (k == "render_split_min") *value = options().render_split_min;
    else return invalid("unknown option '" + k + "'");
    return IVRGS_OK;
}

int64_t ivrgs_edit_table_floats(int32_t n_models) { return (int64_t)IVRGS_EDIT_STRIDE * n_models + 12; }

ivrgs_status ivrgs_compose_edit(const ivrgs_gaussians* models, int32_t n_models, const ivrgs_model_edit* edits,
                                const ivrgs_light* light, ivrgs_gaussians* composed, float* d_edit_table,
                                void* stream) {
    set_error("");
    if (n_models < 1 || n_models > IVRGS_MAX_MODELS)
        return invalid("n_models must be in [1, " + std::to_string(IVRGS_MAX_MODELS) + "]");
    if (!edits || !light || !d_edit_table) return invalid("edits, light and d_edit_table must be non-NULL");
    if (!aligned(d_edit_table, 4)) return invalid("d_edit_table misaligned");
    for (int m = 0; m < n_models; ++m)
        if (!isfinite(edits[m].opacity_scale)) return invalid("non-finite opacity_scale");
    cudaStream_t s = (cudaStream_t)stream;
    if (composed) {
        if (!models) return invalid("models is NULL while composed is given");
        ivrgs_status st = check_gaussians(composed, "composed", true);
        if (st) return st;
        long long total = 0;
        for (int m = 0; m < n_models; ++m) {
            if ((st = check_gaussians(&models[m], "models[m]", false))) return st;
            total += models[m].n;
        }
        if (total != composed->n)
            return invalid("composed->n = " + std::to_string(composed->n) + " but the models hold " +
                           std::to_string(total));
        if (composed->n_models != n_models) return invalid("composed->n_models must equal n_models");
        if ((st = cuda_status(launch_compose(models, n_models, composed, s), "ivrgs_compose_edit"))) return st;
    }
    return cuda_status(launch_edit_table(edits, n_models, light, d_edit_table, s), "ivrgs_compose_edit");
}

ivrgs_status ivrgs_project(const ivrgs_gaussians* g, const float* d_edit_table, const ivrgs_camera* cams,
                           int32_t n_views, float lowpass, ivrgs_projected* out, void* stream) {
    set_error("");
    ivrgs_status st = check_gaussians(g, "g", true, true);
    if (st) return st;
    if (g->n_models < 1 || g->n_models > IVRGS_MAX_MODELS) return invalid("g->n_models out of range");
    if (!d_edit_table) return invalid("d_edit_table is NULL");
    if (!(lowpass >= 0.f) || !isfinite(lowpass)) return invalid("lowpass must be finite and >= 0");
    static thread_local CamBatch cb;
    if ((st = make_cam_batch(cams, n_views, &cb))) return st;
    if ((st = check_projected(out, g->n, n_views))) return st;
    return cuda_status(launch_project(g, d_edit_table, cb, lowpass, out, (cudaStream_t)stream), "ivrgs_project");
}

ivrgs_status ivrgs_morton_keys(const ivrgs_gaussians* g, const float* lo, const float* hi, uint64_t* d_keys,
                               void* stream) {
    set_error("");
    ivrgs_status st = check_gaussians(g, "g", true);
    if (st) return st;
    if (!lo || !hi || (!d_keys && g->n > 0)) return invalid("lo, hi and d_keys must be non-NULL");
    for (int k = 0; k < 3; ++k)
        if (!(hi[k] > lo[k]) || !isfinite(lo[k]) || !isfinite(hi[k])) return invalid("the box needs lo < hi, finite");
    if (!aligned(d_keys, 8)) return invalid("d_keys must be 8-byte aligned");
    return cuda_status(launch_morton(g, lo, hi, d_keys, (cudaStream_t)stream), "ivrgs_morton_keys");
}

ivrgs_status ivrgs_pack_mixed(const ivrgs_gaussians* in, const uint32_t* d_order, ivrgs_gaussians* out,
                              void* stream) {
    set_error("");
    ivrgs_status st = check_gaussians(in, "in", true);
    if (st) return st;
    if (!out) return invalid("out is NULL");
    if (out->precision != IVRGS_MIXED) return invalid("out->precision must be IVRGS_MIXED");
    if ((st = check_gaussians(out, "out", true, true))) return st;
    if (out->n != in->n) return invalid("out->n must equal in->n");
    if (d_order && !aligned(d_order, 4)) return invalid("d_order misaligned");
    return cuda_status(launch_pack_mixed(in, d_order, out, (cudaStream_t)stream), "ivrgs_pack_mixed");
}

ivrgs_status ivrgs_bin_workspace(int64_t n, int32_t n_views, const ivrgs_camera* cams, int32_t tile_w,
                                 int32_t tile_h, int64_t capacity, size_t* bytes) {
    set_error("");
    if (!bytes) return invalid("bytes is NULL");
    if (tile_w != kTile || !tile_height_ok(tile_h)) {
        set_error("tiles are 16 pixels wide and 16 or 8 high");
        return IVRGS_ERR_UNSUPPORTED;
    }
    if (n < 0 || capacity < 0 || capacity >= IVRGS_MAX_PAIRS) return invalid("bad n or capacity");
    static thread_local CamBatch cb;
    ivrgs_status st = make_cam_batch(cams, n_views, &cb, tile_h);
    if (st) return st;
    if (n * (long long)n_views >= IVRGS_MAX_PAIRS) return invalid("n * n_views must be below 2^30 for binning");
    *bytes = plan_bin(n * (long long)n_views, cb.n_tiles, capacity).total_bytes;
    return IVRGS_OK;
}

// error flag of a bin workspace: bit 0 = a look-back wait gave up, bit 1 = the emission wrote a
// different number of pairs than the count pass reported
static ivrgs_status bin_flag_status(unsigned flag) {
    if (flag & 1u) {
        set_error("radix sort look-back wait exceeded its bound");
        return IVRGS_ERR_TIMEOUT;
    }
    if (flag & 2u) {
        set_error("tile emission disagreed with the pair count");
        return IVRGS_ERR_CUDA;
    }
    return IVRGS_OK;
}

ivrgs_status ivrgs_bin(const ivrgs_projected* p, const ivrgs_camera* cams, int32_t n_views, int32_t mode,
                       void* d_workspace, size_t ws_bytes, ivrgs_bins* out, void* stream) {
    set_error("");
    static thread_local CamBatch cb;
    ivrgs_status st = make_cam_batch(cams, n_views, &cb, out ? out->tile_h : kTile);
    if (st) return st;
    if (!p) return invalid("projected is NULL");
    if ((st = check_projected(p, p->n, n_views))) return st;
    if ((st = check_bins(out, cb))) return st;
    if (mode & ~(IVRGS_BIN_CAPACITY | IVRGS_BIN_CULL))
        return invalid("mode must be IVRGS_BIN_EXACT or IVRGS_BIN_CAPACITY, optionally | IVRGS_BIN_CULL");
    const int cull = (mode & IVRGS_BIN_CULL) ? 1 : 0;
    const bool capacity_mode = (mode & IVRGS_BIN_CAPACITY) != 0;
    // the radix look-back carries 30-bit counts, so the records of one call stay below 2^30
    if (p->n * (long long)n_views >= IVRGS_MAX_PAIRS) return invalid("n * n_views must be below 2^30 for binning");
    const BinPlan plan = plan_bin(p->n * (long long)n_views, cb.n_tiles, out->capacity);
    if (!d_workspace || ws_bytes < plan.total_bytes) {
        set_error("workspace too small: need " + std::to_string(plan.total_bytes) + " bytes");
        return IVRGS_ERR_CAPACITY;
    }
    if (!aligned(d_workspace, 256)) return invalid("workspace must be 256-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    char* ws = static_cast<char*>(d_workspace);
    if ((st = cuda_status(launch_bin_count(p, cb, plan, cull, ws, out->d_n_pairs, s), "ivrgs_bin count"))) return st;
    long long exact = -1;
    if (!capacity_mode) {
        unsigned long long total = 0;
        if ((st = cuda_status(cudaMemcpyAsync(&total, out->d_n_pairs, 8, cudaMemcpyDeviceToHost, s), "ivrgs_bin")))
            return st;
        if ((st = cuda_status(cudaStreamSynchronize(s), "ivrgs_bin"))) return st;
        out->n_pairs = (int64_t)total;
        if ((long long)total > out->capacity) {
            set_error("capacity " + std::to_string(out->capacity) + " < " + std::to_string(total) + " pairs");
            return IVRGS_ERR_CAPACITY;
        }
        exact = (long long)total;
    }
    if ((st = cuda_status(launch_bin_sort(p, cb, plan, cull, ws, out, exact, s), "ivrgs_bin sort"))) return st;
    if (!capacity_mode) {
        unsigned flag = 0;
        if ((st = cuda_status(cudaMemcpyAsync(&flag, ws + plan.off_flag, 4, cudaMemcpyDeviceToHost, s), "ivrgs_bin")))
            return st;
        if ((st = cuda_status(cudaStreamSynchronize(s), "ivrgs_bin"))) return st;
        return bin_flag_status(flag);
    }
    return IVRGS_OK;
}

ivrgs_status ivrgs_bin_check(const void* d_workspace, void* stream) {
    set_error("");
    if (!d_workspace) return invalid("workspace is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned flag = 0;  // the flag is the first word of every bin workspace
    ivrgs_status st;
    if ((st = cuda_status(cudaMemcpyAsync(&flag, d_workspace, 4, cudaMemcpyDeviceToHost, s), "ivrgs_bin_check")))
        return st;
    if ((st = cuda_status(cudaStreamSynchronize(s), "ivrgs_bin_check"))) return st;
    return bin_flag_status(flag);
}

ivrgs_status ivrgs_render(const ivrgs_projected* p, const ivrgs_bins* b, const ivrgs_camera* cams, int32_t n_views,
                          const float* bg, float* d_rgba, float* d_final_T, uint32_t* d_last, void* stream) {
    set_error("");
    static thread_local CamBatch cb;
    ivrgs_status st = make_cam_batch(cams, n_views, &cb, b ? b->tile_h : kTile);
    if (st) return st;
    if (!p) return invalid("projected is NULL");
    if ((st = check_projected(p, p->n, n_views))) return st;
    if ((st = check_bins(b, cb))) return st;
    if (!bg || !d_rgba || !d_final_T || !d_last) return invalid("bg and output arrays must be non-NULL");
    if (!aligned(d_rgba, 16)) return invalid("d_rgba must be 16-byte aligned");
    return cuda_status(launch_render(p, b, cb, bg, d_rgba, d_final_T, d_last, (cudaStream_t)stream), "ivrgs_render");
}

ivrgs_status ivrgs_render_aux(const ivrgs_gaussians* g, const float* d_edit_table, const ivrgs_projected* p,
                              const ivrgs_bins* b, const ivrgs_camera* cams, int32_t n_views, float* d_aux,
                              void* stream) {
    set_error("");
    static thread_local CamBatch cb;
    ivrgs_status st = make_cam_batch(cams, n_views, &cb, b ? b->tile_h : kTile);
    if (st) return st;
    if ((st = check_gaussians(g, "g", true, true))) return st;
    if (g->n_models < 1 || g->n_models > IVRGS_MAX_MODELS) return invalid("g->n_models out of range");
    if (!p) return invalid("projected is NULL");
    if (p->n != g->n) return invalid("p->n must equal g->n");
    if ((st = check_projected(p, p->n, n_views))) return st;
    if ((st = check_bins(b, cb))) return st;
    if (!d_edit_table || !d_aux) return invalid("d_edit_table and d_aux must be non-NULL");
    if (!aligned(d_aux, 16)) return invalid("d_aux must be 16-byte aligned");
    return cuda_status(launch_render_aux(g, d_edit_table, p, b, cb, d_aux, (cudaStream_t)stream), "ivrgs_render_aux");
}

ivrgs_status ivrgs_render_aux_backward_workspace(int64_t n, int32_t n_views, size_t* bytes) {
    set_error("");
    if (!bytes || n < 0 || n_views < 1 || n_views > IVRGS_MAX_VIEWS) return invalid("bad arguments");
    *bytes = aux_backward_workspace(n, n_views);
    return IVRGS_OK;
}

ivrgs_status ivrgs_render_aux_backward(const ivrgs_gaussians* g, const float* d_edit_table, const ivrgs_projected* p,
                                       const ivrgs_bins* b, const ivrgs_camera* cams, int32_t n_views, float lowpass,
                                       const float* d_final_T, const uint32_t* d_last, const float* d_dL_daux,
                                       void* d_workspace, size_t ws_bytes, ivrgs_gaussians* grad, float* d_edit_grad,
                                       void* stream) {
    set_error("");
    ivrgs_status st = check_gaussians(g, "g", true, true);
    if (st) return st;
    if (g->n_models < 1 || g->n_models > IVRGS_MAX_MODELS) return invalid("g->n_models out of range");
    if ((st = check_gaussians(grad, "grad", false))) return st;
    if (grad->n != g->n) return invalid("grad->n must equal g->n");
    if (g->sh && (!grad->sh || grad->sh_degree != g->sh_degree))
        return invalid("g has SH colour: grad->sh must be set, with the same sh_degree");
    static thread_local CamBatch cb;
    if ((st = make_cam_batch(cams, n_views, &cb, b ? b->tile_h : kTile))) return st;
    if (!p) return invalid("projected is NULL");
    if ((st = check_projected(p, g->n, n_views))) return st;
    if ((st = check_bins(b, cb))) return st;
    if (!d_edit_table || !d_final_T || !d_last || !d_dL_daux || !d_edit_grad)
        return invalid("NULL input/output array");
    if (!aligned(d_dL_daux, 16)) return invalid("d_dL_daux must be 16-byte aligned");
    if (!(lowpass >= 0.f) || !isfinite(lowpass)) return invalid("lowpass must be finite and >= 0");
    const size_t need = aux_backward_workspace(g->n, n_views);
    if (!d_workspace || ws_bytes < need) {
        set_error("workspace too small: need " + std::to_string(need) + " bytes");
        return IVRGS_ERR_CAPACITY;
    }
    if (!aligned(d_workspace, 256)) return invalid("workspace must be 256-byte aligned");
    return cuda_status(launch_render_aux_backward(g, d_edit_table, p, b, cb, lowpass, d_final_T, d_last, d_dL_daux,
                                                  static_cast<char*>(d_workspace), grad, d_edit_grad,
                                                  (cudaStream_t)stream),
                       "ivrgs_render_aux_backward");
}

ivrgs_status ivrgs_render_backward_workspace(int64_t n, int32_t n_views, size_t* bytes) {
    set_error("");
    if (!bytes || n < 0 || n_views < 1 || n_views > IVRGS_MAX_VIEWS) return invalid("bad arguments");
    *bytes = (size_t)n * (size_t)n_views * 36 + 256;
    return IVRGS_OK;
}

static ivrgs_status render_backward_impl(int accumulate, const ivrgs_gaussians* g, const float* d_edit_table, const ivrgs_projected* p,
                                   const ivrgs_bins* b, const ivrgs_camera* cams, int32_t n_views, float lowpass,
                                   const float* bg, const float* d_final_T, const uint32_t* d_last,
                                   const float* d_dL_drgba, void* d_workspace, size_t ws_bytes,
                                   ivrgs_gaussians* grad, float* d_edit_grad, void* stream) {
    set_error("");
    ivrgs_status st = check_gaussians(g, "g", true, true);
    if (st) return st;
    if (g->n_models < 1 || g->n_models > IVRGS_MAX_MODELS) return invalid("g->n_models out of range");
    if ((st = check_gaussians(grad, "grad", false))) return st;
    if (grad->n != g->n) return invalid("grad->n must equal g->n");
    if (g->sh && (!grad->sh || grad->sh_degree != g->sh_degree))
        return invalid("g has SH colour: grad->sh must be set, with the same sh_degree");
    static thread_local CamBatch cb;
    if ((st = make_cam_batch(cams, n_views, &cb, b ? b->tile_h : kTile))) return st;
    if ((st = check_projected(p, g->n, n_views))) return st;
    if ((st = check_bins(b, cb))) return st;
    if (!d_edit_table || !bg || !d_final_T || !d_last || !d_dL_drgba || !d_edit_grad)
        return invalid("NULL input/output array");
    if (!aligned(d_dL_drgba, 16)) return invalid("d_dL_drgba must be 16-byte aligned");
    if (!(lowpass >= 0.f) || !isfinite(lowpass)) return invalid("lowpass must be finite and >= 0");
    size_t need = 0;
    ivrgs_render_backward_workspace(g->n, n_views, &need);
    if (!d_workspace || ws_bytes < need) {
        set_error("workspace too small: need " + std::to_string(need) + " bytes");
        return IVRGS_ERR_CAPACITY;
    }
    if (!aligned(d_workspace, 256)) return invalid("workspace must be 256-byte aligned");
    return cuda_status(launch_render_backward(g, d_edit_table, p, b, cb, lowpass, bg, d_final_T, d_last, d_dL_drgba,
                                              static_cast<char*>(d_workspace), grad, d_edit_grad, accumulate,
                                              (cudaStream_t)stream),
                       "ivrgs_render_backward");
}

ivrgs_status ivrgs_render_backward(const ivrgs_gaussians* g, const float* d_edit_table, const ivrgs_projected* p,
                                   const ivrgs_bins* b, const ivrgs_camera* cams, int32_t n_views, float lowpass,
                                   const float* bg, const float* d_final_T, const uint32_t* d_last,
                                   const float* d_dL_drgba, void* d_workspace, size_t ws_bytes,
                                   ivrgs_gaussians* grad, float* d_edit_grad, void* stream) {
    return render_backward_impl(0, g, d_edit_table, p, b, cams, n_views, lowpass, bg, d_final_T, d_last, d_dL_drgba,
                                d_workspace, ws_bytes, grad, d_edit_grad, stream);
}

ivrgs_status ivrgs_render_backward_accumulate(const ivrgs_gaussians* g, const float* d_edit_table,
                                              const ivrgs_projected* p, const ivrgs_bins* b, const ivrgs_camera* cams,
                                              int32_t n_views, float lowpass, const float* bg, const float* d_final_T,
                                              const uint32_t* d_last, const float* d_dL_drgba, void* d_workspace,
                                              size_t ws_bytes, ivrgs_gaussians* grad, float* d_edit_grad,
                                              void* stream) {
    return render_backward_impl(1, g, d_edit_table, p, b, cams, n_views, lowpass, bg, d_final_T, d_last, d_dL_drgba,
                                d_workspace, ws_bytes, grad, d_edit_grad, stream);
}

}  // extern "C"

// ------------------------------------------------------------------------- inverse exploration
static long long packed_pixels(const CamBatch& cb) {
    long long n = 0;
    for (int v = 0; v < cb.n; ++v) n = std::max(n, cb.c[v].pix0 + (long long)cb.c[v].W * cb.c[v].H);
    return n;
}

ivrgs_status ivrgs_image_loss_workspace(const ivrgs_camera* cams, int32_t n_views, size_t* bytes) {
    set_error("");
    if (!bytes) return invalid("bytes is NULL");
    static thread_local CamBatch cb;
    ivrgs_status st = make_cam_batch(cams, n_views, &cb);
    if (st) return st;
    *bytes = image_loss_workspace(cb, packed_pixels(cb));
    return IVRGS_OK;
}

ivrgs_status ivrgs_image_loss(const float* d_rgba, const float* d_target, const ivrgs_camera* cams, int32_t n_views,
                              float lambda_ssim, void* d_workspace, size_t ws_bytes, float* d_loss,
                              float* d_dL_drgba, void* stream) {
    set_error("");
    static thread_local CamBatch cb;
    ivrgs_status st = make_cam_batch(cams, n_views, &cb);
    if (st) return st;
    if (!d_rgba || !d_target || !d_loss || !d_dL_drgba) return invalid("device arrays must be non-NULL");
    if (!aligned(d_rgba, 16) || !aligned(d_target, 16) || !aligned(d_dL_drgba, 16))
        return invalid("d_rgba, d_target and d_dL_drgba must be 16-byte aligned");
    if (!(lambda_ssim >= 0.0f && lambda_ssim <= 1.0f)) return invalid("lambda_ssim must be in [0, 1]");
    const long long n_pix = packed_pixels(cb);
    const size_t need = image_loss_workspace(cb, n_pix);
    if (!d_workspace || ws_bytes < need) {
        set_error("workspace too small: need " + std::to_string(need) + " bytes");
        return IVRGS_ERR_CAPACITY;
    }
    if (!aligned(d_workspace, 256)) return invalid("workspace must be 256-byte aligned");
    return cuda_status(launch_image_loss(d_rgba, d_target, cb, n_pix, lambda_ssim, static_cast<char*>(d_workspace),
                                         d_loss, d_dL_drgba, (cudaStream_t)stream),
                       "ivrgs_image_loss");
}

int64_t ivrgs_edit_adam_state_floats(int32_t n_models) { return 2ll * (4ll * n_models + 10) + 3; }

ivrgs_status ivrgs_edit_adam_init(const float* d_edit_table, int32_t n_models, float* d_state, void* stream) {
    set_error("");
    if (n_models < 1 || n_models > IVRGS_MAX_MODELS) return invalid("n_models out of range");
    if (!d_edit_table || !d_state) return invalid("device arrays must be non-NULL");
    return cuda_status(launch_edit_adam_init(d_edit_table, n_models, d_state, (cudaStream_t)stream),
                       "ivrgs_edit_adam_init");
}

ivrgs_status ivrgs_edit_adam(float* d_edit_table, const float* d_edit_grad, int32_t n_models, float* d_state,
                             int32_t learn, float lr, float beta1, float beta2, float eps, void* stream) {
    set_error("");
    if (n_models < 1 || n_models > IVRGS_MAX_MODELS) return invalid("n_models out of range");
    if (!d_edit_table || !d_edit_grad || !d_state) return invalid("device arrays must be non-NULL");
    if (learn & ~(IVRGS_LEARN_COLOR | IVRGS_LEARN_OPACITY | IVRGS_LEARN_LIGHT_MAGNITUDE | IVRGS_LEARN_LIGHT_DIRECTION))
        return invalid("unknown bits in learn");
    if (!(lr > 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return invalid("need lr > 0, 0 <= beta1, beta2 < 1, eps > 0");
    return cuda_status(launch_edit_adam(d_edit_table, d_edit_grad, n_models, d_state, learn, lr, beta1, beta2, eps,
                                        (cudaStream_t)stream),
                       "ivrgs_edit_adam");
}

// ------------------------------------------------------------------------- vector quantisation
ivrgs_status ivrgs_vq_build_workspace(int32_t n_models, int32_t k, size_t* bytes) {
    set_error("");
    if (!bytes) return invalid("bytes is NULL");
    if (n_models < 1 || n_models > IVRGS_MAX_MODELS) return invalid("n_models out of range");
    if (k < 1 || k > IVRGS_VQ_MAX_K) return invalid("k must be in [1, IVRGS_VQ_MAX_K]");
    *bytes = vq_workspace(n_models, k);
    return IVRGS_OK;
}

ivrgs_status ivrgs_vq_build(const ivrgs_gaussians* src, int32_t k, int32_t iters, ivrgs_gaussians* out,
                            void* d_workspace, size_t ws_bytes, void* stream) {
    set_error("");
    ivrgs_status st = check_gaussians(src, "src", true);
    if (st) return st;
    if (src->n_models < 1 || src->n_models > IVRGS_MAX_MODELS) return invalid("src->n_models out of range");
    if (k < 1 || k > IVRGS_VQ_MAX_K) return invalid("k must be in [1, IVRGS_VQ_MAX_K]");
    if (iters < 0) return invalid("iters must be >= 0");
    if (!out) return invalid("out is NULL");
    if (out->precision != IVRGS_VQ || out->n != src->n || out->n_models != src->n_models || out->vq_k != k)
        return invalid("out must be IVRGS_VQ with the n, n_models of src and vq_k = k");
    if (src->n > 0 && (!out->log_scale || !out->quat || !out->opacity_logit || !out->dcolor || !out->kads))
        return invalid("out: NULL index array");
    if (!out->codebook || !aligned(out->codebook, 4)) return invalid("out: codebook NULL or misaligned");
    if (src->n > 0 && (!aligned(out->quat, 4) || !aligned(out->kads, 4)))
        return invalid("out: quat and kads index arrays must be 4-byte aligned");
    const size_t need = vq_workspace(src->n_models, k);
    if (!d_workspace || ws_bytes < need) {
        set_error("workspace too small: need " + std::to_string(need) + " bytes");
        return IVRGS_ERR_CAPACITY;
    }
    if (!aligned(d_workspace, 256)) return invalid("workspace must be 256-byte aligned");
    return cuda_status(launch_vq_build(src, k, iters, out, static_cast<char*>(d_workspace), (cudaStream_t)stream),
                       "ivrgs_vq_build");
}

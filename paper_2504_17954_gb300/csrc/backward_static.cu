// ivrgs_render_backward_static: the backward without a caller-provided workspace.
//
// Its scratch (the per-(view, Gaussian) gradients of the 2D quantities) lives in the
// file-scope device array below, which every GPU that loads the library keeps until the
// process exits. The host never dereferences the array's name: on the first call on each
// device the device address is looked up with cudaGetSymbolAddress (with that device
// current) and cached together with the CUDA context it belongs to; a call under another
// context (after cudaDeviceReset, or a context the caller created) looks it up again. That
// address is handed to the regular backward entry point.
#include <mutex>
#include <string>

#include "common.cuh"

namespace ivrgs {

constexpr size_t kStaticScratchBytes = (size_t)IVRGS_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_bwd_scratch[kStaticScratchBytes];

static std::mutex g_scratch_mu;
static void* g_scratch_ptr[kMaxDevices] = {};
static void* g_scratch_ctx[kMaxDevices] = {};

// The calling thread's current CUDA context (the driver's cuCtxGetCurrent, reached through the
// runtime's entry-point query so that the library needs no link-time driver dependency); NULL
// when none is current or the query is unavailable.
static void* current_context() {
    typedef int (*CtxGetCurrent)(void**);
    static CtxGetCurrent fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<CtxGetCurrent>(f);
    }();
    void* ctx = nullptr;
    if (!fn || fn(&ctx) != 0) return nullptr;
    return ctx;
}

static ivrgs_status scratch_address(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "ivrgs_render_backward_static: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("ivrgs_render_backward_static: device ordinal " + std::to_string(dev) + " out of range");
        return IVRGS_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    void* ctx = current_context();
    if (!g_scratch_ptr[dev] || !ctx || ctx != g_scratch_ctx[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_bwd_scratch);  // also makes the device's context current
        if (e != cudaSuccess) return cuda_status(e, "ivrgs_render_backward_static: cudaGetSymbolAddress");
        g_scratch_ptr[dev] = p;
        g_scratch_ctx[dev] = ctx ? ctx : current_context();
    }
    *out = g_scratch_ptr[dev];
    return IVRGS_OK;
}

}  // namespace ivrgs

using namespace ivrgs;

extern "C" ivrgs_status ivrgs_render_backward_static(const ivrgs_gaussians* g, const float* d_edit_table,
                                                     const ivrgs_projected* p, const ivrgs_bins* b,
                                                     const ivrgs_camera* cams, int32_t n_views, float lowpass,
                                                     const float* bg, const float* d_final_T, const uint32_t* d_last,
                                                     const float* d_dL_drgba, ivrgs_gaussians* grad,
                                                     float* d_edit_grad, void* stream) {
    set_error("");
    if (!g) {
        set_error("g is NULL");
        return IVRGS_ERR_INVALID_ARG;
    }
    size_t need = 0;
    ivrgs_status st = ivrgs_render_backward_workspace(g->n, n_views, &need);
    if (st) return st;
    if (need > kStaticScratchBytes) {
        set_error("ivrgs_render_backward_static: n * n_views = " + std::to_string(g->n * (long long)n_views) +
                  " needs " + std::to_string(need) + " bytes of scratch but the built-in array holds " +
                  std::to_string(kStaticScratchBytes) + "; use ivrgs_render_backward with a workspace");
        return IVRGS_ERR_CAPACITY;
    }
    void* scratch = nullptr;
    if ((st = scratch_address(&scratch))) return st;
    return ivrgs_render_backward(g, d_edit_table, p, b, cams, n_views, lowpass, bg, d_final_T, d_last, d_dL_drgba,
                                 scratch, kStaticScratchBytes, grad, d_edit_grad, stream);
}

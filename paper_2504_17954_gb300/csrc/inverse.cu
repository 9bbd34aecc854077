// Inverse volume exploration (Sec. 4.6): the image loss between a rendering and a reference
// image, and one optimiser step on the edit parameters.
//
// Loss: (1 - lambda) L1 + lambda (1 - SSIM) over the RGB channels of every view (the 3DGS loss
// the paper's "combination of L1 and SSIM" refers to), with L1 = mean |x - y| and SSIM the mean
// of the per-pixel, per-channel structural similarity with an 11 x 11 Gaussian window
// (sigma 1.5, weights normalised), C1 = 0.01^2, C2 = 0.03^2, and zero padding at each view's
// border. Per pixel q and channel, with mu = w * x, E[x^2] = w * x^2 etc. (w * = windowed sum):
//   S = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2)),
//   s_x^2 = E[x^2] - mu_x^2, s_xy = E[xy] - mu_x mu_y.
// Its gradient w.r.t. x_p is sum_q w(q - p) (dS/dmu_x(q) + 2 x_p dS/ds_x^2(q) + y_p dS/ds_xy(q))
// with dS/dmu_x the total derivative at fixed E[.]; the window is symmetric, so each sum is one
// more blur of a per-pixel map. Every blur is separable (a horizontal and a vertical 11-tap pass).
//
// Optimiser: Adam (Kingma and Ba) on the learnable slots of the edit table (c_p and the opacity
// scale of every model, lambda, b) and on the global light's polar and azimuthal angles
// (dir = (sin t cos p, sin t sin p, cos t)), with the step counter kept on the device so that a
// captured CUDA graph can replay whole iterations.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace ivrgs {

constexpr int kSsimR = 5;  // window radius (11 taps)
constexpr float kSsimC1 = 0.01f * 0.01f, kSsimC2 = 0.03f * 0.03f;
constexpr int kLossThreads = 256;

struct SsimWin {
    float w[2 * kSsimR + 1];
};

// normalised 1D Gaussian weights (sigma 1.5); the 2D window is their outer product
static SsimWin ssim_window() {
    SsimWin s;
    double t[2 * kSsimR + 1], sum = 0.0;
    for (int k = -kSsimR; k <= kSsimR; ++k) {
        t[k + kSsimR] = std::exp(-(double)(k * k) / (2.0 * 1.5 * 1.5));
        sum += t[k + kSsimR];
    }
    for (int k = 0; k < 2 * kSsimR + 1; ++k) s.w[k] = (float)(t[k] / sum);
    return s;
}

// ------------------------------------------------------------------------- forward passes
// pass 1, horizontal: per channel (x, y, x^2, y^2, xy) windowed along the row -> h1 [pix][15]
__global__ void __launch_bounds__(kLossThreads) k_ssim_h1(const float4* __restrict__ x, const float4* __restrict__ y,
                                                          const __grid_constant__ CamBatch cb, SsimWin win,
                                                          float* __restrict__ h1) {
    const CamDev& c = cb.c[blockIdx.y];
    const long long q = (long long)blockIdx.x * kLossThreads + threadIdx.x;
    if (q >= (long long)c.W * c.H) return;
    const int i = (int)(q % c.W), j = (int)(q / c.W);
    float acc[15];
#pragma unroll
    for (int k = 0; k < 15; ++k) acc[k] = 0.f;
    const long long row = c.pix0 + (long long)j * c.W;
#pragma unroll
    for (int k = -kSsimR; k <= kSsimR; ++k) {
        const int ii = i + k;
        if (ii < 0 || ii >= c.W) continue;
        const float wk = win.w[k + kSsimR];
        const float4 a = x[row + ii], b = y[row + ii];
        const float xa[3] = {a.x, a.y, a.z}, yb[3] = {b.x, b.y, b.z};
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            acc[5 * ch + 0] += wk * xa[ch];
            acc[5 * ch + 1] += wk * yb[ch];
            acc[5 * ch + 2] += wk * xa[ch] * xa[ch];
            acc[5 * ch + 3] += wk * yb[ch] * yb[ch];
            acc[5 * ch + 4] += wk * xa[ch] * yb[ch];
        }
    }
    float* o = h1 + 15 * (c.pix0 + q);
#pragma unroll
    for (int k = 0; k < 15; ++k) o[k] = acc[k];
}

__device__ __forceinline__ float block_sum(float v, float* s_red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int w = 0; w < kLossThreads / 32; ++w) t += s_red[w];
    __syncthreads();
    return t;
}

// pass 2, vertical: the windowed moments, the SSIM value and, scaled by dL/dS = -lambda / N,
// the maps (dS/dmu_x total, dS/ds_x^2, dS/ds_xy) -> d1 [pix][9]; block sums of S and |x - y|
__global__ void __launch_bounds__(kLossThreads) k_ssim_v1(const float4* __restrict__ x, const float4* __restrict__ y,
                                                          const float* __restrict__ h1,
                                                          const __grid_constant__ CamBatch cb, SsimWin win, float gS,
                                                          float* __restrict__ d1, double* __restrict__ part) {
    __shared__ float s_red[kLossThreads / 32];
    const CamDev& c = cb.c[blockIdx.y];
    const long long q = (long long)blockIdx.x * kLossThreads + threadIdx.x;
    float ssum = 0.f, l1 = 0.f;
    if (q < (long long)c.W * c.H) {
        const int i = (int)(q % c.W), j = (int)(q / c.W);
        float m[15];
#pragma unroll
        for (int k = 0; k < 15; ++k) m[k] = 0.f;
#pragma unroll
        for (int k = -kSsimR; k <= kSsimR; ++k) {
            const int jj = j + k;
            if (jj < 0 || jj >= c.H) continue;
            const float wk = win.w[k + kSsimR];
            const float* hp = h1 + 15 * (c.pix0 + (long long)jj * c.W + i);
#pragma unroll
            for (int t = 0; t < 15; ++t) m[t] += wk * hp[t];
        }
        const float4 a = x[c.pix0 + q], b = y[c.pix0 + q];
        const float xa[3] = {a.x, a.y, a.z}, yb[3] = {b.x, b.y, b.z};
        float* o = d1 + 9 * (c.pix0 + q);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float mx = m[5 * ch], my = m[5 * ch + 1];
            const float sx = m[5 * ch + 2] - mx * mx, sy = m[5 * ch + 3] - my * my, sxy = m[5 * ch + 4] - mx * my;
            const float A1 = 2.f * mx * my + kSsimC1, A2 = 2.f * sxy + kSsimC2;
            const float B1 = mx * mx + my * my + kSsimC1, B2 = sx + sy + kSsimC2;
            const float iB = 1.f / (B1 * B2);
            const float S = A1 * A2 * iB;
            const float dmu = 2.f * my * A2 * iB - S * 2.f * mx / B1;  // at fixed sigmas
            const float dsx = -S / B2;
            const float dsxy = 2.f * A1 * iB;
            // total derivative in mu_x at fixed E[x^2], E[xy]
            o[3 * ch + 0] = gS * (dmu - 2.f * mx * dsx - my * dsxy);
            o[3 * ch + 1] = gS * dsx;
            o[3 * ch + 2] = gS * dsxy;
            ssum += S;
            l1 += fabsf(xa[ch] - yb[ch]);
        }
    }
    const long long pb = (long long)blockIdx.y * gridDim.x + blockIdx.x;
    const float ts = block_sum(ssum, s_red);
    const float tl = block_sum(l1, s_red);
    if (threadIdx.x == 0) {
        part[2 * pb] = ts;
        part[2 * pb + 1] = tl;
    }
}

// pass 3, horizontal blur of the 9 derivative maps -> h2 [pix][9]
__global__ void __launch_bounds__(kLossThreads) k_ssim_h2(const float* __restrict__ d1,
                                                          const __grid_constant__ CamBatch cb, SsimWin win,
                                                          float* __restrict__ h2) {
    const CamDev& c = cb.c[blockIdx.y];
    const long long q = (long long)blockIdx.x * kLossThreads + threadIdx.x;
    if (q >= (long long)c.W * c.H) return;
    const int i = (int)(q % c.W), j = (int)(q / c.W);
    float acc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = 0.f;
    const long long row = c.pix0 + (long long)j * c.W;
#pragma unroll
    for (int k = -kSsimR; k <= kSsimR; ++k) {
        const int ii = i + k;
        if (ii < 0 || ii >= c.W) continue;
        const float wk = win.w[k + kSsimR];
        const float* dp = d1 + 9 * (row + ii);
#pragma unroll
        for (int t = 0; t < 9; ++t) acc[t] += wk * dp[t];
    }
    float* o = h2 + 9 * (c.pix0 + q);
#pragma unroll
    for (int k = 0; k < 9; ++k) o[k] = acc[k];
}

// pass 4, vertical blur and the pixel gradient: dL/dx = B0 + 2 x B1 + y B2 + (1 - lambda) sign(x - y) / N
__global__ void __launch_bounds__(kLossThreads) k_ssim_v2(const float4* __restrict__ x, const float4* __restrict__ y,
                                                          const float* __restrict__ h2,
                                                          const __grid_constant__ CamBatch cb, SsimWin win, float gL1,
                                                          float4* __restrict__ dL) {
    const CamDev& c = cb.c[blockIdx.y];
    const long long q = (long long)blockIdx.x * kLossThreads + threadIdx.x;
    if (q >= (long long)c.W * c.H) return;
    const int i = (int)(q % c.W), j = (int)(q / c.W);
    float B[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) B[k] = 0.f;
#pragma unroll
    for (int k = -kSsimR; k <= kSsimR; ++k) {
        const int jj = j + k;
        if (jj < 0 || jj >= c.H) continue;
        const float wk = win.w[k + kSsimR];
        const float* hp = h2 + 9 * (c.pix0 + (long long)jj * c.W + i);
#pragma unroll
        for (int t = 0; t < 9; ++t) B[t] += wk * hp[t];
    }
    const float4 a = x[c.pix0 + q], b = y[c.pix0 + q];
    const float xa[3] = {a.x, a.y, a.z}, yb[3] = {b.x, b.y, b.z};
    float g[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const float d = xa[ch] - yb[ch];
        const float s = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        g[ch] = B[3 * ch] + 2.f * xa[ch] * B[3 * ch + 1] + yb[ch] * B[3 * ch + 2] + gL1 * s;
    }
    dL[c.pix0 + q] = make_float4(g[0], g[1], g[2], 0.f);
}

// lambda = 0 (the plain L1 loss): dL/dx = sign(x - y) / N per colour channel and the block
// sums of |x - y|, without the SSIM passes (the SSIM block sums are written as 0)
__global__ void __launch_bounds__(kLossThreads) k_l1_loss(const float4* __restrict__ x, const float4* __restrict__ y,
                                                          const __grid_constant__ CamBatch cb, float gL1,
                                                          float4* __restrict__ dL, double* __restrict__ part) {
    __shared__ float s_red[kLossThreads / 32];
    const CamDev& c = cb.c[blockIdx.y];
    const long long q = (long long)blockIdx.x * kLossThreads + threadIdx.x;
    float l1 = 0.f;
    if (q < (long long)c.W * c.H) {
        const float4 a = x[c.pix0 + q], b = y[c.pix0 + q];
        const float d[3] = {a.x - b.x, a.y - b.y, a.z - b.z};
        float g[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            g[ch] = d[ch] > 0.f ? gL1 : (d[ch] < 0.f ? -gL1 : 0.f);
            l1 += fabsf(d[ch]);
        }
        dL[c.pix0 + q] = make_float4(g[0], g[1], g[2], 0.f);
    }
    const long long pb = (long long)blockIdx.y * gridDim.x + blockIdx.x;
    const float tl = block_sum(l1, s_red);
    if (threadIdx.x == 0) {
        part[2 * pb] = 0.0;
        part[2 * pb + 1] = tl;
    }
}

__global__ void k_loss_final(const double* __restrict__ part, long long n_part, double n_elems, float lambda,
                             float* __restrict__ loss) {
    __shared__ double s_s[256], s_l[256];
    double a = 0.0, b = 0.0;
    for (long long k = threadIdx.x; k < n_part; k += 256) {
        a += part[2 * k];
        b += part[2 * k + 1];
    }
    s_s[threadIdx.x] = a;
    s_l[threadIdx.x] = b;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s_s[threadIdx.x] += s_s[threadIdx.x + o];
            s_l[threadIdx.x] += s_l[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double ssim = s_s[0] / n_elems, l1 = s_l[0] / n_elems;
        loss[0] = (float)((1.0 - lambda) * l1 + lambda * (1.0 - ssim));
        loss[1] = (float)l1;
        loss[2] = (float)ssim;
    }
}

static long long max_view_pixels(const CamBatch& cb) {
    long long m = 0;
    for (int v = 0; v < cb.n; ++v) m = std::max(m, (long long)cb.c[v].W * cb.c[v].H);
    return m;
}

size_t image_loss_workspace(const CamBatch& cb, long long n_pix) {
    const long long bx = (max_view_pixels(cb) + kLossThreads - 1) / kLossThreads;
    const size_t maps = (size_t)n_pix * (15 + 9 + 9) * sizeof(float);
    return ((maps + 255) & ~size_t(255)) + sizeof(double) * 2 * (size_t)(bx * cb.n);
}

cudaError_t launch_image_loss(const float* rgba, const float* target, const CamBatch& cb, long long n_pix,
                              float lambda, char* ws, float* loss, float* dL, cudaStream_t s) {
    const long long bx = (max_view_pixels(cb) + kLossThreads - 1) / kLossThreads;
    if (bx == 0) return cudaSuccess;
    long long n_elems = 0;
    for (int v = 0; v < cb.n; ++v) n_elems += 3ll * cb.c[v].W * cb.c[v].H;
    float* h1 = reinterpret_cast<float*>(ws);
    float* d1 = h1 + 15 * n_pix;
    float* h2 = d1 + 9 * n_pix;
    const size_t maps = (size_t)n_pix * (15 + 9 + 9) * sizeof(float);
    double* part = reinterpret_cast<double*>(ws + ((maps + 255) & ~size_t(255)));
    const SsimWin win = ssim_window();
    const dim3 grid((unsigned)bx, (unsigned)cb.n);
    const float4* x = reinterpret_cast<const float4*>(rgba);
    const float4* y = reinterpret_cast<const float4*>(target);
    const float gS = -lambda / (float)n_elems, gL1 = (1.0f - lambda) / (float)n_elems;
    if (lambda == 0.0f) {
        IVRGS_PROF("k_l1_loss", s);
        k_l1_loss<<<grid, kLossThreads, 0, s>>>(x, y, cb, gL1, reinterpret_cast<float4*>(dL), part);
        k_loss_final<<<1, 256, 0, s>>>(part, bx * cb.n, (double)n_elems, lambda, loss);
    } else {
        IVRGS_PROF("k_image_loss", s);
        k_ssim_h1<<<grid, kLossThreads, 0, s>>>(x, y, cb, win, h1);
        k_ssim_v1<<<grid, kLossThreads, 0, s>>>(x, y, h1, cb, win, gS, d1, part);
        k_ssim_h2<<<grid, kLossThreads, 0, s>>>(d1, cb, win, h2);
        k_ssim_v2<<<grid, kLossThreads, 0, s>>>(x, y, h2, cb, win, gL1, reinterpret_cast<float4*>(dL));
        k_loss_final<<<1, 256, 0, s>>>(part, bx * cb.n, (double)n_elems, lambda, loss);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------- Adam
// state: m[P], v[P], then (polar, azimuth), then the step count t (as a float); P = 4 M + 8 + 2
__global__ void __launch_bounds__(1024) k_edit_adam(float* __restrict__ table, const float* __restrict__ egrad,
                                                    int n_models, float* __restrict__ state, int flags, float lr,
                                                    float b1, float b2, float eps) {
    const int M = n_models, P = 4 * M + 8 + 2;
    float* m = state;
    float* v = state + P;
    float* ang = state + 2 * P;
    float* tstep = state + 2 * P + 2;
    const float t = tstep[0] + 1.0f;
    const float bc1 = 1.0f - powf(b1, t), bc2 = 1.0f - powf(b2, t);
    const float th = ang[0], ph = ang[1];
    float* L = table + (long long)M * IVRGS_EDIT_STRIDE + 8;
    __syncthreads();
    for (int j = threadIdx.x; j < P; j += blockDim.x) {
        float g, *param = nullptr;
        bool learn;
        if (j < 4 * M) {
            const int mm = j >> 2, k = j & 3;
            param = table + (long long)mm * IVRGS_EDIT_STRIDE + k;
            g = egrad[(long long)mm * IVRGS_EDIT_STRIDE + k];
            learn = (k < 3 ? (flags & IVRGS_LEARN_COLOR) : (flags & IVRGS_LEARN_OPACITY)) != 0;
        } else if (j < 4 * M + 8) {
            const int k = j - 4 * M;
            param = table + (long long)M * IVRGS_EDIT_STRIDE + k;
            g = egrad[(long long)M * IVRGS_EDIT_STRIDE + k];
            learn = (flags & IVRGS_LEARN_LIGHT_MAGNITUDE) != 0;
        } else {
            // d/d angle of dir(polar, azimuth) = sum_k dL/d dir_k d dir_k / d angle
            const float* gd = egrad + (long long)M * IVRGS_EDIT_STRIDE + 8;
            const float st = sinf(th), ct = cosf(th), sp = sinf(ph), cp = cosf(ph);
            g = j == 4 * M + 8 ? gd[0] * ct * cp + gd[1] * ct * sp - gd[2] * st : -gd[0] * st * sp + gd[1] * st * cp;
            learn = (flags & IVRGS_LEARN_LIGHT_DIRECTION) != 0 && L[3] != 0.0f;
        }
        if (!learn) continue;
        const float mj = b1 * m[j] + (1.0f - b1) * g;
        const float vj = b2 * v[j] + (1.0f - b2) * g * g;
        m[j] = mj;
        v[j] = vj;
        const float step = lr * (mj / bc1) / (sqrtf(vj / bc2) + eps);
        if (param) *param -= step;
        else ang[j - (4 * M + 8)] -= step;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        tstep[0] = t;
        if ((flags & IVRGS_LEARN_LIGHT_DIRECTION) && L[3] != 0.0f) {
            const float a = ang[0], b = ang[1];
            L[0] = sinf(a) * cosf(b);
            L[1] = sinf(a) * sinf(b);
            L[2] = cosf(a);
        }
    }
}

// zero moments and step; angles of the table's global light (polar from +z, azimuth from +x)
__global__ void k_edit_adam_init(const float* __restrict__ table, int n_models, float* __restrict__ state) {
    const int P = 4 * n_models + 8 + 2;
    for (int j = threadIdx.x; j < 2 * P + 3; j += blockDim.x) state[j] = 0.0f;
    __syncthreads();
    if (threadIdx.x == 0) {
        const float* L = table + (long long)n_models * IVRGS_EDIT_STRIDE + 8;
        const float r = sqrtf(L[0] * L[0] + L[1] * L[1] + L[2] * L[2]);
        state[2 * P] = r > 0.0f ? acosf(fminf(fmaxf(L[2] / r, -1.0f), 1.0f)) : 0.0f;
        state[2 * P + 1] = atan2f(L[1], L[0]);
    }
}

cudaError_t launch_edit_adam_init(const float* table, int n_models, float* state, cudaStream_t s) {
    k_edit_adam_init<<<1, 1024, 0, s>>>(table, n_models, state);
    return cudaGetLastError();
}

cudaError_t launch_edit_adam(float* table, const float* egrad, int n_models, float* state, int flags, float lr,
                             float b1, float b2, float eps, cudaStream_t s) {
    IVRGS_PROF("k_edit_adam", s);
    k_edit_adam<<<1, 1024, 0, s>>>(table, egrad, n_models, state, flags, lr, b1, b2, eps);
    return cudaGetLastError();
}

}  // namespace ivrgs

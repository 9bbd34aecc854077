/*
 * ivrgs_oracle.c -- plain, slow CPU reference of the editable-Gaussian rasterizer.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is checked against.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may load it; the
 * product library never does.  It shares no code with the CUDA path.
 *
 * Everything is float64 and scalar, written in the order of the paper's definitions:
 *   Sec. 3 (Preliminaries), first equation: Gaussian G(x) = exp(-1/2 (x-mu)^T Sigma^-1 (x-mu)),
 *     Sigma from a quaternion q and a scale s; projected covariance Sigma' = J W Sigma W^T J^T.
 *   Sec. 3, second equation: C = sum_i T_i alpha_i c_i, T_i = prod_{j<i} (1 - alpha_j),
 *     alpha = Gaussian weight times opacity.
 *   Sec. 3, Blinn-Phong system: c = k_a I_a + k_d I_d |n.l| + [|n.l|>0] k_s I_s |n.h|^beta,
 *     I_a = I_d = c_v, I_s = white, h = (v+l)/|v+l|.
 *   Sec. 4.3: c_v = c_p + dc (palette colour per basic model plus per-Gaussian offset).
 *   Sec. 4.5: composition = concatenation of the basic models; colour edit replaces c_p;
 *     opacity edit scales the opacity; light edits scale {k_a,k_d,k_s,beta}.
 *   Sec. 4.6: light magnitude as lambda*{k_a,k_d,k_s,beta} + b (global), light direction.
 *
 * Where the paper is silent the 3DGS lineage it builds on fixes the rest (stated as named
 * parameters): opacity = sigmoid(logit), scale = exp(log s), a low-pass dilation delta*I of
 * Sigma', a 1.3x guard band on x/z and y/z inside J, a near plane, radius = ceil(3 sqrt(
 * lambda_max)), 16x16 tiles, alpha clamped at 0.99, contributions with alpha < 1/255 skipped,
 * and the walk stopping before a Gaussian that would take the transmittance below 1e-4.
 *
 * Integer decisions that the GPU takes in float32 (tile rectangle, sort key) are taken here
 * in float32 too, from the float64 values rounded once: the rectangle from (u, v) rounded
 * to float and the integer radius; the key from the bit pattern of the float64 camera depth
 * z = (R mu + t)_z rounded once to float32.  The near-plane decision compares the float64 z
 * with z_near.
 *
 * Gradients (reverse mode of all of the above) are taken w.r.t. the stored parameters:
 * mean, log-scale, unnormalised quaternion and normal, opacity logit, colour offset,
 * (k_a,k_d,k_s,beta), and the edit parameters {c_p, opacity scale} per model, {lambda, b}
 * global, and the orbital light direction: per view, or the edit table's global light
 * direction when that is switched on (Sec. 4.6 learns one light direction for the composed
 * model, as polar and azimuthal angles).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t W, H;
    double fx, fy, cx, cy;
    double R[9];      /* world -> camera rotation, row-major */
    double t[3];
    double campos[3];
    double znear;
    int32_t headlight; /* 1: light at the camera (l = v); 0: directional light_dir */
    double light_dir[3];
} orc_camera;

typedef struct {
    int64_t n;
    const double *mean, *log_scale, *quat, *opacity_logit, *dcolor, *normal, *kads;
    const int32_t* model_id;
    const double* sh; /* NULL: Blinn-Phong colour; else [n][(deg+1)^2][3] SH coefficients */
    int32_t sh_deg;
} orc_gaussians;

/* Real spherical harmonics up to degree 3 (the view-dependent colour of 3DGS that Sec. 3 and
   Sec. 4.2 refer to), orthonormal on the unit sphere, with the Condon-Shortley sign: on a unit
   direction (x, y, z), Y_0 = 1/(2 sqrt(pi)); degree 1: -a y, a z, -a x (a = sqrt(3/(4 pi)));
   degree 2: b xy, -b yz, c (2z^2 - x^2 - y^2), -b xz, e (x^2 - y^2) (b = sqrt(15/(4 pi)),
   c = sqrt(5/(16 pi)), e = sqrt(15/(16 pi))); degree 3: -f y(3x^2 - y^2), g xyz,
   -h y(4z^2 - x^2 - y^2), k z(2z^2 - 3x^2 - 3y^2), -h x(4z^2 - x^2 - y^2), m z(x^2 - y^2),
   -f x(x^2 - 3y^2) (f = sqrt(35/(32 pi)), g = sqrt(105/(4 pi)), h = sqrt(21/(32 pi)),
   k = sqrt(7/(16 pi)), m = sqrt(105/(16 pi))). Y[k] and the gradient dY[k] w.r.t. (x, y, z)
   (the polynomials differentiated as written). */
static void sh_basis(const double d[3], int deg, double Y[16], double dY[16][3]) {
    const double PI = 3.14159265358979323846;
    const double x = d[0], y = d[1], z = d[2];
    const double Y0 = 0.5 / sqrt(PI), a = sqrt(3.0 / (4 * PI)), b = sqrt(15.0 / (4 * PI)),
                 c = sqrt(5.0 / (16 * PI)), e = sqrt(15.0 / (16 * PI)), f = sqrt(35.0 / (32 * PI)),
                 g = sqrt(105.0 / (4 * PI)), h = sqrt(21.0 / (32 * PI)), k = sqrt(7.0 / (16 * PI)),
                 m = sqrt(105.0 / (16 * PI));
    memset(Y, 0, 16 * sizeof(double));
    memset(dY, 0, 16 * 3 * sizeof(double));
    Y[0] = Y0;
    if (deg < 1) return;
    Y[1] = -a * y; dY[1][1] = -a;
    Y[2] = a * z;  dY[2][2] = a;
    Y[3] = -a * x; dY[3][0] = -a;
    if (deg < 2) return;
    Y[4] = b * x * y;  dY[4][0] = b * y; dY[4][1] = b * x;
    Y[5] = -b * y * z; dY[5][1] = -b * z; dY[5][2] = -b * y;
    Y[6] = c * (2 * z * z - x * x - y * y); dY[6][0] = -2 * c * x; dY[6][1] = -2 * c * y; dY[6][2] = 4 * c * z;
    Y[7] = -b * x * z; dY[7][0] = -b * z; dY[7][2] = -b * x;
    Y[8] = e * (x * x - y * y); dY[8][0] = 2 * e * x; dY[8][1] = -2 * e * y;
    if (deg < 3) return;
    Y[9] = -f * y * (3 * x * x - y * y);  dY[9][0] = -6 * f * x * y; dY[9][1] = -f * (3 * x * x - 3 * y * y);
    Y[10] = g * x * y * z; dY[10][0] = g * y * z; dY[10][1] = g * x * z; dY[10][2] = g * x * y;
    Y[11] = -h * y * (4 * z * z - x * x - y * y);
    dY[11][0] = 2 * h * x * y; dY[11][1] = -h * (4 * z * z - x * x - 3 * y * y); dY[11][2] = -8 * h * y * z;
    Y[12] = k * z * (2 * z * z - 3 * x * x - 3 * y * y);
    dY[12][0] = -6 * k * x * z; dY[12][1] = -6 * k * y * z; dY[12][2] = k * (6 * z * z - 3 * x * x - 3 * y * y);
    Y[13] = -h * x * (4 * z * z - x * x - y * y);
    dY[13][0] = -h * (4 * z * z - 3 * x * x - y * y); dY[13][1] = 2 * h * x * y; dY[13][2] = -8 * h * x * z;
    Y[14] = m * z * (x * x - y * y); dY[14][0] = 2 * m * x * z; dY[14][1] = -2 * m * y * z; dY[14][2] = m * (x * x - y * y);
    Y[15] = -f * x * (x * x - 3 * y * y); dY[15][0] = -f * (3 * x * x - 3 * y * y); dY[15][1] = 6 * f * x * y;
}

/* exported for the basis pins: Y[16] and dY[16][3] at direction d (unit) */
void orc_sh_basis(const double* d, int32_t deg, double* Y, double* dY) {
    sh_basis(d, deg, Y, (double(*)[3])dY);
}

/* edit table: per model m: [c_p(3), opacity scale, visible, 0, 0, 0]; then lambda(4), b(4),
   global light (l_x, l_y, l_z, on): with on != 0 every view with an orbital light uses
   l / |l| instead of its own light_dir */
#define EDIT_STRIDE 8

static const double* table_light(const double* edit, int32_t n_models) {
    const double* L = edit + (int64_t)n_models * EDIT_STRIDE + 8;
    return L[3] != 0.0 ? L : NULL;
}

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static double norm3(const double* a) { return sqrt(dot3(a, a)); }

static double sgn(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0); }

/* rotation matrix of the normalised quaternion (w, x, y, z) */
static void quat_rot(const double* q, double* qn, double R[9]) {
    double len = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double w = q[0] / len, x = q[1] / len, y = q[2] / len, z = q[3] / len;
    qn[0] = w; qn[1] = x; qn[2] = y; qn[3] = z;
    R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z);       R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);       R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);       R[7] = 2.0 * (y * z + w * x);       R[8] = 1.0 - 2.0 * (x * x + y * y);
}

/* dR/dq (normalised components), dRdq[k][i] = d R_i / d qn_k */
static void quat_rot_jac(const double* qn, double d[4][9]) {
    double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    double dw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
    double dx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
    double dy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
    double dz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
    memcpy(d[0], dw, sizeof dw); memcpy(d[1], dx, sizeof dx);
    memcpy(d[2], dy, sizeof dy); memcpy(d[3], dz, sizeof dz);
}

/* ---------------------------------------------------------------------------------------
 * Per-Gaussian forward quantities for one view (everything the blend and the backward use)
 * --------------------------------------------------------------------------------------- */
typedef struct {
    int visible;          /* 0: culled */
    double mc[3];         /* camera-space mean */
    double Sig[9];        /* 3D covariance */
    double M[9];          /* R_q S */
    double Rq[9], qn[4];
    double S[3];          /* exp(log s) */
    double txc, tyc;      /* clamped x/z, y/z */
    int clampx, clampy;
    double J[6], T[6];    /* J (2x3), T = J W (2x3) */
    double cov[3];        /* Sigma' entries A, B, C */
    double det;
    double conic[3];      /* a, b, c */
    double lmax;
    int32_t radius;
    double radius_margin;
    double uv[2];
    double depth;
    double depth_margin;  /* distance of z to the nearest float32 rounding midpoint / (|t2| + sum |R2k mk|) */
    /* shading */
    double sig_o, opacity;
    double cv[3], kp[4];
    double vdir[3], vlen;     /* v = (campos - mu)/|.|, |campos - mu| */
    double l[3];
    double hv[3], hlen, h[3];
    double nn[3], nlen;
    double ndl, ndh, nl, nh;
    int gate;
    double spec_pow;
    double rgb[3];
    int sh_on;               /* SH colour (3DGS) instead of Blinn-Phong */
    double sdir[3], sdlen;   /* (mu - campos) / |.|, |mu - campos| */
    double Ysh[16], dYsh[16][3];
    int sh_clamp[3];         /* raw SH colour + 0.5 < 0: clamped to 0 */
} orc_fwd;

static void project_one(const orc_gaussians* G, int64_t g, const double* edit, int32_t n_models,
                        const orc_camera* cam, double lowpass, double guard, orc_fwd* f) {
    memset(f, 0, sizeof *f);
    int32_t m = G->model_id[g];
    const double* me = edit + (int64_t)m * EDIT_STRIDE;
    const double* lam = edit + (int64_t)n_models * EDIT_STRIDE;
    const double* bias = lam + 4;
    const double* mu = G->mean + 3 * g;
    const double* R = cam->R;
    if (me[4] == 0.0) return; /* model hidden (Sec. 4.5 selection of basic models) */
    /* viewing transform W: mu_c = R mu + t */
    for (int i = 0; i < 3; ++i) f->mc[i] = R[3 * i] * mu[0] + R[3 * i + 1] * mu[1] + R[3 * i + 2] * mu[2] + cam->t[i];
    double x = f->mc[0], y = f->mc[1], z = f->mc[2];
    f->depth = z;
    {   /* how close z lies to a point where its rounding to float32 changes (for certification) */
        double mag = fabs(cam->t[2]) + fabs(R[6] * mu[0]) + fabs(R[7] * mu[1]) + fabs(R[8] * mu[2]);
        float z32 = (float)z;
        double lo = 0.5 * ((double)z32 + (double)nextafterf(z32, -INFINITY));
        double hi = 0.5 * ((double)z32 + (double)nextafterf(z32, INFINITY));
        double d = fabs(z - lo) < fabs(z - hi) ? fabs(z - lo) : fabs(z - hi);
        f->depth_margin = mag > 0.0 ? d / mag : d;
    }
    if (!(z > cam->znear)) return; /* behind the near plane */
    /* Sigma = R_q S S^T R_q^T */
    quat_rot(G->quat + 4 * g, f->qn, f->Rq);
    for (int k = 0; k < 3; ++k) f->S[k] = exp(G->log_scale[3 * g + k]);
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) f->M[3 * i + k] = f->Rq[3 * i + k] * f->S[k];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += f->M[3 * i + k] * f->M[3 * j + k];
            f->Sig[3 * i + j] = s;
        }
    /* Jacobian of the perspective map at the (guard-band clamped) mean */
    double limx = guard * (0.5 * cam->W) / cam->fx, limy = guard * (0.5 * cam->H) / cam->fy;
    double tx = x / z, ty = y / z;
    f->txc = tx; f->tyc = ty;
    if (tx < -limx) { f->txc = -limx; f->clampx = 1; }
    if (tx > limx) { f->txc = limx; f->clampx = 1; }
    if (ty < -limy) { f->tyc = -limy; f->clampy = 1; }
    if (ty > limy) { f->tyc = limy; f->clampy = 1; }
    f->J[0] = cam->fx / z; f->J[1] = 0.0; f->J[2] = -cam->fx * f->txc / z;
    f->J[3] = 0.0; f->J[4] = cam->fy / z; f->J[5] = -cam->fy * f->tyc / z;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += f->J[3 * i + k] * R[3 * k + j];
            f->T[3 * i + j] = s;
        }
    /* Sigma' = T Sigma T^T + delta I */
    double cv2[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double s = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) s += f->T[3 * i + a] * f->Sig[3 * a + b] * f->T[3 * j + b];
            cv2[2 * i + j] = s;
        }
    f->cov[0] = cv2[0] + lowpass;
    f->cov[1] = cv2[1];
    f->cov[2] = cv2[3] + lowpass;
    f->det = f->cov[0] * f->cov[2] - f->cov[1] * f->cov[1];
    if (!(f->det > 0.0)) return;
    f->conic[0] = f->cov[2] / f->det;
    f->conic[1] = -f->cov[1] / f->det;
    f->conic[2] = f->cov[0] / f->det;
    double mid = 0.5 * (f->cov[0] + f->cov[2]);
    double disc = mid * mid - f->det;
    f->lmax = mid + sqrt(disc > 0.0 ? disc : 0.0);
    double r3 = 3.0 * sqrt(f->lmax);
    f->radius = (int32_t)ceil(r3);
    double fr = r3 - floor(r3);
    f->radius_margin = (fr < 1.0 - fr ? fr : 1.0 - fr) / (r3 > 1.0 ? r3 : 1.0);
    if (f->radius <= 0) return;
    f->uv[0] = cam->fx * (x / z) + cam->cx;
    f->uv[1] = cam->fy * (y / z) + cam->cy;
    /* editable opacity (Sec. 4.5): o' = s_m sigmoid(logit), not clamped */
    f->sig_o = sigmoid(G->opacity_logit[g]);
    f->opacity = me[3] * f->sig_o;
    /* Blinn-Phong colour of the Gaussian (Sec. 3 with the edits of Sec. 4.3-4.6) */
    for (int c = 0; c < 3; ++c) f->cv[c] = me[c] + G->dcolor[3 * g + c];
    for (int k = 0; k < 4; ++k) f->kp[k] = lam[k] * G->kads[4 * g + k] + bias[k];
    double d[3] = {cam->campos[0] - mu[0], cam->campos[1] - mu[1], cam->campos[2] - mu[2]};
    f->vlen = norm3(d);
    for (int c = 0; c < 3; ++c) f->vdir[c] = d[c] / f->vlen;
    if (cam->headlight) {
        for (int c = 0; c < 3; ++c) f->l[c] = f->vdir[c];
    } else {
        const double* L = table_light(edit, n_models);
        const double* ld = L ? L : cam->light_dir;
        double ll = norm3(ld);
        for (int c = 0; c < 3; ++c) f->l[c] = ld[c] / ll;
    }
    for (int c = 0; c < 3; ++c) f->hv[c] = f->vdir[c] + f->l[c];
    f->hlen = norm3(f->hv);
    for (int c = 0; c < 3; ++c) f->h[c] = f->hlen > 0.0 ? f->hv[c] / f->hlen : 0.0;
    const double* n = G->normal + 3 * g;
    f->nlen = norm3(n);
    for (int c = 0; c < 3; ++c) f->nn[c] = n[c] / f->nlen;
    f->ndl = dot3(f->nn, f->l);
    f->ndh = dot3(f->nn, f->h);
    f->nl = fabs(f->ndl);
    f->nh = fabs(f->ndh);
    f->gate = (f->nl > 0.0 && f->nh > 0.0);
    f->spec_pow = f->gate ? pow(f->nh, f->kp[3]) : 0.0;
    for (int c = 0; c < 3; ++c)
        f->rgb[c] = f->kp[0] * f->cv[c] + f->kp[1] * f->nl * f->cv[c] + (f->gate ? f->kp[2] * f->spec_pow : 0.0);
    if (G->sh) { /* 3DGS colour: SH of the direction from the camera, + 0.5, clamped at 0 */
        f->sh_on = 1;
        f->sdlen = f->vlen;
        for (int c = 0; c < 3; ++c) f->sdir[c] = -f->vdir[c];
        sh_basis(f->sdir, G->sh_deg, f->Ysh, f->dYsh);
        const int nb = (G->sh_deg + 1) * (G->sh_deg + 1);
        const double* shg = G->sh + (int64_t)g * nb * 3;
        for (int c = 0; c < 3; ++c) {
            double v = 0.5;
            for (int kk = 0; kk < nb; ++kk) v += shg[3 * kk + c] * f->Ysh[kk];
            f->sh_clamp[c] = v < 0.0;
            f->rgb[c] = v < 0.0 ? 0.0 : v;
        }
    }
    f->visible = 1;
}

/* Project all Gaussians for one view.  radius[g] == 0 marks a culled Gaussian. */
void orc_project(int64_t n, const double* mean, const double* log_scale, const double* quat,
                 const double* opacity_logit, const double* dcolor, const double* normal,
                 const double* kads, const int32_t* model_id, const double* sh, int32_t sh_deg,
                 const double* edit, int32_t n_models,
                 const orc_camera* cam, double lowpass, double guard,
                 double* uv, double* cov, double* conic, double* opacity, double* rgb,
                 double* depth, int32_t* radius, double* radius_margin, double* depth_margin) {
    orc_gaussians G = {n, mean, log_scale, quat, opacity_logit, dcolor, normal, kads, model_id, sh, sh_deg};
    orc_fwd f;
    for (int64_t g = 0; g < n; ++g) {
        project_one(&G, g, edit, n_models, cam, lowpass, guard, &f);
        radius[g] = f.visible ? f.radius : 0;
        radius_margin[g] = f.radius_margin;
        uv[2 * g] = f.uv[0]; uv[2 * g + 1] = f.uv[1];
        for (int c = 0; c < 3; ++c) {
            cov[3 * g + c] = f.cov[c];
            conic[3 * g + c] = f.conic[c];
            rgb[3 * g + c] = f.rgb[c];
        }
        opacity[g] = f.opacity;
        depth[g] = f.depth;
        depth_margin[g] = f.depth_margin;
    }
}

/* ---------------------------------------------------------------------------------------
 * Tile binning and ordering.  Decision inputs are float32: (u, v), the integer radius and
 * the float32 depth.  Rectangle (half-open tile ranges):
 *   x0 = clamp(floor((u - r)/Tw), 0, Gx), x1 = clamp(floor((u + r)/Tw) + 1, 0, Gx)
 * and the same for y.  Key = (global tile << 32) | bits(depth); ties keep the emission order
 * (view, Gaussian index), i.e. the sort is stable.
 * --------------------------------------------------------------------------------------- */
static void rect32(float u, float v, int32_t r, int32_t gx, int32_t gy, int32_t tw, int32_t th, int32_t* rc) {
    float fr = (float)r;
    float a = floorf((u - fr) / (float)tw), b = floorf((u + fr) / (float)tw) + 1.0f;
    float c = floorf((v - fr) / (float)th), d = floorf((v + fr) / (float)th) + 1.0f;
    a = fminf(fmaxf(a, 0.0f), (float)gx); b = fminf(fmaxf(b, 0.0f), (float)gx);
    c = fminf(fmaxf(c, 0.0f), (float)gy); d = fminf(fmaxf(d, 0.0f), (float)gy);
    rc[0] = (int32_t)a; rc[1] = (int32_t)b; rc[2] = (int32_t)c; rc[3] = (int32_t)d;
}

typedef struct { uint64_t key; int64_t seq; uint32_t value; } orc_pair;

static int pair_cmp(const void* pa, const void* pb) {
    const orc_pair* a = (const orc_pair*)pa;
    const orc_pair* b = (const orc_pair*)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->seq < b->seq ? -1 : (a->seq > b->seq ? 1 : 0);
}

/* Returns the number of pairs.  Writes keys/values/ranges only if it is <= capacity.
   tile_offset[V+1] receives the first global tile of each view. */
int64_t orc_bin(int32_t n_views, int64_t n, const float* uv, const int32_t* radius, const float* depth,
                const int32_t* Ws, const int32_t* Hs, int32_t tw, int32_t th,
                uint64_t* keys, uint32_t* values, int64_t capacity, uint32_t* ranges, int64_t* tile_offset) {
    tile_offset[0] = 0;
    for (int v = 0; v < n_views; ++v) {
        int64_t gx = (Ws[v] + tw - 1) / tw, gy = (Hs[v] + th - 1) / th;
        tile_offset[v + 1] = tile_offset[v] + gx * gy;
    }
    int64_t total = 0;
    int32_t rc[4];
    for (int v = 0; v < n_views; ++v) {
        int32_t gx = (Ws[v] + tw - 1) / tw, gy = (Hs[v] + th - 1) / th;
        for (int64_t g = 0; g < n; ++g) {
            int64_t i = (int64_t)v * n + g;
            if (radius[i] <= 0) continue;
            rect32(uv[2 * i], uv[2 * i + 1], radius[i], gx, gy, tw, th, rc);
            total += (int64_t)(rc[1] - rc[0]) * (rc[3] - rc[2]);
        }
    }
    if (total > capacity) return total;
    orc_pair* P = (orc_pair*)malloc(sizeof(orc_pair) * (size_t)(total > 0 ? total : 1));
    int64_t k = 0;
    for (int v = 0; v < n_views; ++v) {
        int32_t gx = (Ws[v] + tw - 1) / tw, gy = (Hs[v] + th - 1) / th;
        for (int64_t g = 0; g < n; ++g) {
            int64_t i = (int64_t)v * n + g;
            if (radius[i] <= 0) continue;
            rect32(uv[2 * i], uv[2 * i + 1], radius[i], gx, gy, tw, th, rc);
            uint32_t bits;
            memcpy(&bits, &depth[i], 4);
            for (int ty = rc[2]; ty < rc[3]; ++ty)
                for (int tx = rc[0]; tx < rc[1]; ++tx) {
                    uint64_t tile = (uint64_t)(tile_offset[v] + (int64_t)ty * gx + tx);
                    P[k].key = (tile << 32) | bits;
                    P[k].seq = k;
                    P[k].value = (uint32_t)g;
                    ++k;
                }
        }
    }
    qsort(P, (size_t)total, sizeof(orc_pair), pair_cmp);
    int64_t nt = tile_offset[n_views];
    memset(ranges, 0, sizeof(uint32_t) * 2 * (size_t)nt);
    for (int64_t i = 0; i < total; ++i) {
        keys[i] = P[i].key;
        values[i] = P[i].value;
        uint64_t t = P[i].key >> 32;
        if (i == 0 || (P[i - 1].key >> 32) != t) ranges[2 * t] = (uint32_t)i;
        if (i == total - 1 || (P[i + 1].key >> 32) != t) ranges[2 * t + 1] = (uint32_t)(i + 1);
    }
    free(P);
    return total;
}

/* The pairs of ONE view whose tile row lies in [row_begin, row_end), ordered as orc_bin orders
   them (by tile, then depth bits, then emission order, i.e. Gaussian index), with global tile
   ids (tile0 = the view's first global tile).  Returns the pair count; writes keys and values
   only if it is <= capacity.  Disjoint row bands concatenated in row order give orc_bin's
   ordering of that view, so bands may be binned concurrently. */
int64_t orc_bin_view_rows(int64_t n, const float* uv, const int32_t* radius, const float* depth, int32_t W,
                          int32_t H, int32_t tw, int32_t th, int64_t tile0, int32_t row_begin, int32_t row_end,
                          uint64_t* keys, uint32_t* values, int64_t capacity) {
    int32_t gx = (W + tw - 1) / tw, gy = (H + th - 1) / th;
    int32_t rc[4];
    int64_t total = 0;
    for (int64_t g = 0; g < n; ++g) {
        if (radius[g] <= 0) continue;
        rect32(uv[2 * g], uv[2 * g + 1], radius[g], gx, gy, tw, th, rc);
        int32_t y0 = rc[2] > row_begin ? rc[2] : row_begin, y1 = rc[3] < row_end ? rc[3] : row_end;
        if (y1 > y0) total += (int64_t)(rc[1] - rc[0]) * (y1 - y0);
    }
    if (total > capacity) return total;
    orc_pair* P = (orc_pair*)malloc(sizeof(orc_pair) * (size_t)(total > 0 ? total : 1));
    int64_t k = 0;
    for (int64_t g = 0; g < n; ++g) {
        if (radius[g] <= 0) continue;
        rect32(uv[2 * g], uv[2 * g + 1], radius[g], gx, gy, tw, th, rc);
        int32_t y0 = rc[2] > row_begin ? rc[2] : row_begin, y1 = rc[3] < row_end ? rc[3] : row_end;
        uint32_t bits;
        memcpy(&bits, &depth[g], 4);
        for (int ty = y0; ty < y1; ++ty)
            for (int tx = rc[0]; tx < rc[1]; ++tx) {
                uint64_t tile = (uint64_t)(tile0 + (int64_t)ty * gx + tx);
                P[k].key = (tile << 32) | bits;
                P[k].seq = k;
                P[k].value = (uint32_t)g;
                ++k;
            }
    }
    qsort(P, (size_t)total, sizeof(orc_pair), pair_cmp);
    for (int64_t i = 0; i < total; ++i) {
        keys[i] = P[i].key;
        values[i] = P[i].value;
    }
    free(P);
    return total;
}

/* ---------------------------------------------------------------------------------------
 * Front-to-back compositing of one pixel over an ordered list (Sec. 3, second equation).
 * margins[0]: smallest |ln(alpha*255)| over evaluated entries (1/255 cut-off);
 * margins[1]: smallest |ln(T'/1e-4)| over evaluated entries (termination);
 * margins[2]: smallest |P| / (|a|dx^2/2 + |b dx dy| + |c|dy^2/2) (the P > 0 guard);
 * margins[3]: smallest |ln(o G / 0.99)| (the 0.99 clamp; matters for gradients only);
 * margins[4]: sum of (k+1) over contributing entries k, margins[5]: sum of (k+1)^2 over the
 *   contributors whose alpha is clamped -- a signature of the contributor set, so that a test
 *   can tell whether a perturbation changed any discrete decision of the pixel.
 * --------------------------------------------------------------------------------------- */
#define N_MARGINS 6
#define ALPHA_MIN (1.0 / 255.0)
#define ALPHA_MAX 0.99
#define T_MIN 1e-4

typedef struct { const double *uv, *conic, *opacity, *rgb; } orc_view_proj;

static void blend_pixel(const orc_view_proj* P, const uint32_t* list, int64_t len, double px, double py,
                        const double* bg, double* out_rgba, double* out_T, uint32_t* out_last, double* margins,
                        /* optional record for the backward */ int64_t* rec_k, double* rec_T, int64_t* rec_n) {
    double C[3] = {0, 0, 0}, T = 1.0;
    uint32_t last = 0;
    double m[N_MARGINS] = {INFINITY, INFINITY, INFINITY, INFINITY, 0.0, 0.0};
    int64_t nrec = 0;
    for (int64_t k = 0; k < len; ++k) {
        uint32_t g = list[k];
        const double* cn = P->conic + 3 * (int64_t)g;
        double dx = P->uv[2 * (int64_t)g] - px, dy = P->uv[2 * (int64_t)g + 1] - py;
        double Pw = -0.5 * (cn[0] * dx * dx + cn[2] * dy * dy) - cn[1] * dx * dy;
        double scale = 0.5 * fabs(cn[0]) * dx * dx + 0.5 * fabs(cn[2]) * dy * dy + fabs(cn[1] * dx * dy);
        if (scale > 0.0) { double r = fabs(Pw) / scale; if (r < m[2]) m[2] = r; }
        if (Pw > 0.0) continue;
        double raw = P->opacity[g] * exp(Pw);
        if (raw > 0.0) {
            double lm = fabs(log(raw / ALPHA_MAX));
            if (lm < m[3]) m[3] = lm;
        }
        double alpha = raw < ALPHA_MAX ? raw : ALPHA_MAX;
        if (alpha > 0.0) { double la = fabs(log(alpha * 255.0)); if (la < m[0]) m[0] = la; }
        if (alpha < ALPHA_MIN) continue;
        double Tn = T * (1.0 - alpha);
        { double lt = fabs(log(Tn / T_MIN)); if (lt < m[1]) m[1] = lt; }
        if (Tn < T_MIN) break;
        if (rec_k) { rec_k[nrec] = k; rec_T[nrec] = T; }
        ++nrec;
        m[4] += (double)(k + 1);
        if (!(raw < ALPHA_MAX)) m[5] += (double)(k + 1) * (double)(k + 1);
        for (int c = 0; c < 3; ++c) C[c] += T * alpha * P->rgb[3 * (int64_t)g + c];
        T = Tn;
        last = (uint32_t)(k + 1);
    }
    for (int c = 0; c < 3; ++c) out_rgba[c] = C[c] + T * bg[c];
    out_rgba[3] = 1.0 - T;
    *out_T = T;
    *out_last = last;
    if (margins) for (int i = 0; i < N_MARGINS; ++i) margins[i] = m[i];
    if (rec_n) *rec_n = nrec;
}

/* Render the tiles [t_begin, t_end) (row-major within the view) of one view from its projected
   records and its slice of the bins. ranges/values are global (all views); tile0 is this view's
   first global tile.  Tiles are independent, so disjoint tile ranges may run concurrently. */
void orc_render_view_tiles(const double* uv, const double* conic, const double* opacity, const double* rgb,
                           const uint32_t* values, const uint32_t* ranges, int64_t tile0,
                           int32_t W, int32_t H, int32_t tw, int32_t th, const double* bg,
                           double* rgba, double* final_T, uint32_t* last, double* margins,
                           int64_t t_begin, int64_t t_end) {
    orc_view_proj P = {uv, conic, opacity, rgb};
    int32_t gx = (W + tw - 1) / tw;
    for (int64_t tl = t_begin; tl < t_end; ++tl) {
        int32_t ty = (int32_t)(tl / gx), tx = (int32_t)(tl % gx);
        int64_t t = tile0 + tl;
        uint32_t s = ranges[2 * t], e = ranges[2 * t + 1];
        for (int32_t j = ty * th; j < (ty + 1) * th && j < H; ++j)
            for (int32_t i = tx * tw; i < (tx + 1) * tw && i < W; ++i) {
                int64_t p = (int64_t)j * W + i;
                blend_pixel(&P, values + s, (int64_t)e - s, i + 0.5, j + 0.5, bg, rgba + 4 * p,
                            final_T + p, last + p, margins ? margins + N_MARGINS * p : NULL, NULL, NULL, NULL);
            }
    }
}

/* Render one view (all of its tiles). */
void orc_render_view(const double* uv, const double* conic, const double* opacity, const double* rgb,
                     const uint32_t* values, const uint32_t* ranges, int64_t tile0,
                     int32_t W, int32_t H, int32_t tw, int32_t th, const double* bg,
                     double* rgba, double* final_T, uint32_t* last, double* margins) {
    int64_t nt = (int64_t)((W + tw - 1) / tw) * ((H + th - 1) / th);
    orc_render_view_tiles(uv, conic, opacity, rgb, values, ranges, tile0, W, H, tw, th, bg, rgba, final_T, last,
                          margins, 0, nt);
}

/* Auxiliary maps (Sec. 4.2 first equation: D, N = sum_i T_i alpha_i {d_i, n_i}; Sec. 4.3: the
   offset-colour and coefficient maps sum_i T_i alpha_i {dc_i, k_i}): per pixel of one view, the
   contributors and their T_i from blend_pixel, alpha_i from the same formula, and
   out[p][a] = sum_i T_i alpha_i aux[g_i][a] for a < na, then out[p][na] = 1 - T_final. */
void orc_render_view_aux(const double* uv, const double* conic, const double* opacity, const double* rgb,
                         const double* aux, int32_t na, const uint32_t* values, const uint32_t* ranges,
                         int64_t tile0, int32_t W, int32_t H, int32_t tw, int32_t th, double* out) {
    orc_view_proj P = {uv, conic, opacity, rgb};
    int32_t gx = (W + tw - 1) / tw, gy = (H + th - 1) / th;
    int64_t maxlen = 1;
    for (int64_t t = 0; t < (int64_t)gx * gy; ++t) {
        int64_t l = (int64_t)ranges[2 * (tile0 + t) + 1] - ranges[2 * (tile0 + t)];
        if (l > maxlen) maxlen = l;
    }
    int64_t* rk = (int64_t*)malloc(sizeof(int64_t) * (size_t)maxlen);
    double* rT = (double*)malloc(sizeof(double) * (size_t)maxlen);
    const double zero_bg[3] = {0.0, 0.0, 0.0};
    for (int32_t ty = 0; ty < gy; ++ty)
        for (int32_t tx = 0; tx < gx; ++tx) {
            int64_t t = tile0 + (int64_t)ty * gx + tx;
            uint32_t s = ranges[2 * t], e = ranges[2 * t + 1];
            for (int32_t j = ty * th; j < (ty + 1) * th && j < H; ++j)
                for (int32_t i = tx * tw; i < (tx + 1) * tw && i < W; ++i) {
                    int64_t p = (int64_t)j * W + i;
                    double rgba[4], Tf, px = i + 0.5, py = j + 0.5;
                    uint32_t last;
                    int64_t nrec = 0;
                    blend_pixel(&P, values + s, (int64_t)e - s, px, py, zero_bg, rgba, &Tf, &last, NULL, rk, rT,
                                &nrec);
                    double* o = out + (int64_t)(na + 1) * p;
                    for (int a = 0; a <= na; ++a) o[a] = 0.0;
                    for (int64_t r = 0; r < nrec; ++r) {
                        uint32_t g = values[s + rk[r]];
                        const double* cn = conic + 3 * (int64_t)g;
                        double dx = uv[2 * (int64_t)g] - px, dy = uv[2 * (int64_t)g + 1] - py;
                        double Pw = -0.5 * (cn[0] * dx * dx + cn[2] * dy * dy) - cn[1] * dx * dy;
                        double raw = opacity[g] * exp(Pw);
                        double alpha = raw < ALPHA_MAX ? raw : ALPHA_MAX;
                        double w = rT[r] * alpha;
                        for (int a = 0; a < na; ++a) o[a] += w * aux[(int64_t)na * g + a];
                    }
                    o[na] = 1.0 - Tf;
                }
        }
    free(rk);
    free(rT);
}

/* Composite a list of pixels, each with its own explicit ordered list (sampled checks). */
void orc_render_pixels(const double* uv, const double* conic, const double* opacity, const double* rgb,
                       int64_t n_px, const double* pxy, const int64_t* list_off, const uint32_t* lists,
                       const double* bg, double* rgba, double* final_T, uint32_t* last, double* margins) {
    orc_view_proj P = {uv, conic, opacity, rgb};
    for (int64_t p = 0; p < n_px; ++p)
        blend_pixel(&P, lists + list_off[p], list_off[p + 1] - list_off[p], pxy[2 * p], pxy[2 * p + 1], bg,
                    rgba + 4 * p, final_T + p, last + p, margins + N_MARGINS * p, NULL, NULL, NULL);
}

/* ---------------------------------------------------------------------------------------
 * Backward of the compositing for one pixel list, accumulating per-Gaussian gradients of
 * (u, v), conic (a, b, c), opacity o' and rgb.  The forward contributions are recomputed and
 * the transmittance in front of each contributor is kept exactly (no division).
 * With S_i = sum_{j>i} T_j alpha_j c_j + T_final bg:
 *   dC/dc_i = T_i alpha_i,  dC/dalpha_i = T_i c_i - S_i/(1 - alpha_i),
 *   dA/dalpha_i = T_final/(1 - alpha_i)  (A = 1 - T_final).
 * --------------------------------------------------------------------------------------- */
static void blend_pixel_backward(const orc_view_proj* P, const uint32_t* list, int64_t len, double px,
                                 double py, const double* bg, const double* dout, int64_t* rk, double* rT,
                                 double* g_uv, double* g_conic, double* g_opacity, double* g_rgb) {
    double rgba[4], Tf;
    uint32_t last;
    int64_t nrec;
    blend_pixel(P, list, len, px, py, bg, rgba, &Tf, &last, NULL, rk, rT, &nrec);
    double S[3] = {Tf * bg[0], Tf * bg[1], Tf * bg[2]};
    for (int64_t r = nrec - 1; r >= 0; --r) {
        uint32_t g = list[rk[r]];
        const double* cn = P->conic + 3 * (int64_t)g;
        const double* c = P->rgb + 3 * (int64_t)g;
        double dx = P->uv[2 * (int64_t)g] - px, dy = P->uv[2 * (int64_t)g + 1] - py;
        double Pw = -0.5 * (cn[0] * dx * dx + cn[2] * dy * dy) - cn[1] * dx * dy;
        double G = exp(Pw);
        double raw = P->opacity[g] * G;
        int clamped = !(raw < ALPHA_MAX);
        double alpha = clamped ? ALPHA_MAX : raw;
        double Ti = rT[r];
        double dalpha = dout[3] * Tf / (1.0 - alpha);
        for (int ch = 0; ch < 3; ++ch) {
            g_rgb[3 * (int64_t)g + ch] += Ti * alpha * dout[ch];
            dalpha += dout[ch] * (Ti * c[ch] - S[ch] / (1.0 - alpha));
        }
        for (int ch = 0; ch < 3; ++ch) S[ch] += Ti * alpha * c[ch];
        if (clamped) continue;
        double dP = dalpha * raw;
        g_opacity[g] += dalpha * G;
        g_uv[2 * (int64_t)g] += dP * (-(cn[0] * dx + cn[1] * dy));
        g_uv[2 * (int64_t)g + 1] += dP * (-(cn[2] * dy + cn[1] * dx));
        g_conic[3 * (int64_t)g] += dP * (-0.5 * dx * dx);
        g_conic[3 * (int64_t)g + 1] += dP * (-dx * dy);
        g_conic[3 * (int64_t)g + 2] += dP * (-0.5 * dy * dy);
    }
}

/* Backward of the tiles [t_begin, t_end) of one view, accumulating (+=) into the per-Gaussian
   record gradients; concurrent tile ranges need gradient buffers of their own. */
void orc_render_view_backward_tiles(const double* uv, const double* conic, const double* opacity,
                                    const double* rgb, const uint32_t* values, const uint32_t* ranges,
                                    int64_t tile0, int32_t W, int32_t H, int32_t tw, int32_t th, const double* bg,
                                    const double* dL_drgba, double* g_uv, double* g_conic, double* g_opacity,
                                    double* g_rgb, int64_t t_begin, int64_t t_end) {
    orc_view_proj P = {uv, conic, opacity, rgb};
    int32_t gx = (W + tw - 1) / tw;
    int64_t maxlen = 1;
    for (int64_t t = t_begin; t < t_end; ++t) {
        int64_t l = (int64_t)ranges[2 * (tile0 + t) + 1] - ranges[2 * (tile0 + t)];
        if (l > maxlen) maxlen = l;
    }
    int64_t* rk = (int64_t*)malloc(sizeof(int64_t) * (size_t)maxlen);
    double* rT = (double*)malloc(sizeof(double) * (size_t)maxlen);
    for (int64_t tl = t_begin; tl < t_end; ++tl) {
        int32_t ty = (int32_t)(tl / gx), tx = (int32_t)(tl % gx);
        int64_t t = tile0 + tl;
        uint32_t s = ranges[2 * t], e = ranges[2 * t + 1];
        for (int32_t j = ty * th; j < (ty + 1) * th && j < H; ++j)
            for (int32_t i = tx * tw; i < (tx + 1) * tw && i < W; ++i) {
                int64_t p = (int64_t)j * W + i;
                const double* d = dL_drgba + 4 * p;
                if (d[0] == 0.0 && d[1] == 0.0 && d[2] == 0.0 && d[3] == 0.0) continue;
                blend_pixel_backward(&P, values + s, (int64_t)e - s, i + 0.5, j + 0.5, bg, d, rk, rT, g_uv,
                                     g_conic, g_opacity, g_rgb);
            }
    }
    free(rk);
    free(rT);
}

void orc_render_view_backward(const double* uv, const double* conic, const double* opacity, const double* rgb,
                              const uint32_t* values, const uint32_t* ranges, int64_t tile0, int32_t W,
                              int32_t H, int32_t tw, int32_t th, const double* bg, const double* dL_drgba,
                              double* g_uv, double* g_conic, double* g_opacity, double* g_rgb) {
    int64_t nt = (int64_t)((W + tw - 1) / tw) * ((H + th - 1) / th);
    orc_render_view_backward_tiles(uv, conic, opacity, rgb, values, ranges, tile0, W, H, tw, th, bg, dL_drgba, g_uv,
                                   g_conic, g_opacity, g_rgb, 0, nt);
}

/* Backward for an explicit pixel set with explicit lists (sampled full-size checks). */
void orc_render_pixels_backward(const double* uv, const double* conic, const double* opacity, const double* rgb,
                                int64_t n_px, const double* pxy, const int64_t* list_off, const uint32_t* lists,
                                const double* bg, const double* dL_drgba, double* g_uv, double* g_conic,
                                double* g_opacity, double* g_rgb) {
    orc_view_proj P = {uv, conic, opacity, rgb};
    int64_t maxlen = 1;
    for (int64_t p = 0; p < n_px; ++p)
        if (list_off[p + 1] - list_off[p] > maxlen) maxlen = list_off[p + 1] - list_off[p];
    int64_t* rk = (int64_t*)malloc(sizeof(int64_t) * (size_t)maxlen);
    double* rT = (double*)malloc(sizeof(double) * (size_t)maxlen);
    for (int64_t p = 0; p < n_px; ++p)
        blend_pixel_backward(&P, lists + list_off[p], list_off[p + 1] - list_off[p], pxy[2 * p], pxy[2 * p + 1],
                             bg, dL_drgba + 4 * p, rk, rT, g_uv, g_conic, g_opacity, g_rgb);
    free(rk);
    free(rT);
}

/* ---------------------------------------------------------------------------------------
 * Backward of projection + shading + edits for one view.  Accumulates (+=) into parameter
 * gradients (same layout as the parameters), the edit-table gradient (same layout as the
 * edit table) and the light-direction gradient of this view.
 * --------------------------------------------------------------------------------------- */
void orc_project_backward(int64_t n, const double* mean, const double* log_scale, const double* quat,
                          const double* opacity_logit, const double* dcolor, const double* normal,
                          const double* kads, const int32_t* model_id, const double* sh, int32_t sh_deg,
                          const double* edit, int32_t n_models,
                          const orc_camera* cam, double lowpass, double guard,
                          const double* g_uv, const double* g_conic, const double* g_opacity, const double* g_rgb,
                          double* d_mean, double* d_log_scale, double* d_quat, double* d_opacity_logit,
                          double* d_dcolor, double* d_normal, double* d_kads, double* d_sh, double* d_edit,
                          double* d_light) {
    orc_gaussians G = {n, mean, log_scale, quat, opacity_logit, dcolor, normal, kads, model_id, sh, sh_deg};
    const double* lam = edit + (int64_t)n_models * EDIT_STRIDE;
    double* d_lam = d_edit + (int64_t)n_models * EDIT_STRIDE;
    double* d_bias = d_lam + 4;
    const double* R = cam->R;
    orc_fwd f;
    for (int64_t g = 0; g < n; ++g) {
        project_one(&G, g, edit, n_models, cam, lowpass, guard, &f);
        if (!f.visible) continue;
        int32_t m = model_id[g];
        const double* me = edit + (int64_t)m * EDIT_STRIDE;
        double* dme = d_edit + (int64_t)m * EDIT_STRIDE;
        double dmu[3] = {0, 0, 0};
        const double* Gr = g_rgb + 3 * g;
        if (f.sh_on) { /* ---- SH colour: coefficients and the view direction ---- */
            const int nb = (sh_deg + 1) * (sh_deg + 1);
            const double* shg = sh + (int64_t)g * nb * 3;
            double* dshg = d_sh + (int64_t)g * nb * 3;
            double dd[3] = {0, 0, 0};
            for (int c = 0; c < 3; ++c) {
                if (f.sh_clamp[c]) continue;
                for (int kk = 0; kk < nb; ++kk) {
                    dshg[3 * kk + c] += Gr[c] * f.Ysh[kk];
                    for (int j = 0; j < 3; ++j) dd[j] += Gr[c] * shg[3 * kk + c] * f.dYsh[kk][j];
                }
            }
            /* dir = (mu - campos) / |mu - campos| */
            double pd = dot3(f.sdir, dd);
            for (int c = 0; c < 3; ++c) dmu[c] += (dd[c] - f.sdir[c] * pd) / f.sdlen;
            goto opacity;
        }
        {
        /* ---- shading ---- */
        double Gc = Gr[0] * f.cv[0] + Gr[1] * f.cv[1] + Gr[2] * f.cv[2];
        double Gs = Gr[0] + Gr[1] + Gr[2];
        double dkp[4] = {Gc, f.nl * Gc, 0.0, 0.0};
        double dnh = 0.0;
        if (f.gate) {
            dkp[2] = Gs * f.spec_pow;
            dkp[3] = Gs * f.kp[2] * f.spec_pow * log(f.nh);
            dnh = Gs * f.kp[2] * f.kp[3] * pow(f.nh, f.kp[3] - 1.0);
        }
        double dnl = f.kp[1] * Gc;
        for (int c = 0; c < 3; ++c) {
            double dcv = (f.kp[0] + f.kp[1] * f.nl) * Gr[c];
            d_dcolor[3 * g + c] += dcv;
            dme[c] += dcv;
        }
        for (int k = 0; k < 4; ++k) {
            d_kads[4 * g + k] += lam[k] * dkp[k];
            d_lam[k] += kads[4 * g + k] * dkp[k];
            d_bias[k] += dkp[k];
        }
        double snl = sgn(f.ndl), snh = sgn(f.ndh);
        double dnn[3], dl[3], dh[3], dv[3] = {0, 0, 0};
        for (int c = 0; c < 3; ++c) {
            dnn[c] = dnl * snl * f.l[c] + dnh * snh * f.h[c];
            dl[c] = dnl * snl * f.nn[c];
            dh[c] = dnh * snh * f.nn[c];
        }
        if (f.hlen > 0.0) {
            double hd = dot3(f.h, dh);
            for (int c = 0; c < 3; ++c) {
                double dhv = (dh[c] - f.h[c] * hd) / f.hlen;
                dv[c] += dhv;
                dl[c] += dhv;
            }
        }
        if (cam->headlight) {
            for (int c = 0; c < 3; ++c) dv[c] += dl[c];
        } else {
            /* gradient w.r.t. the direction actually used: the table's or the view's */
            const double* L = table_light(edit, n_models);
            const double* lsrc = L ? L : cam->light_dir;
            double* dst = L ? d_edit + (int64_t)n_models * EDIT_STRIDE + 8 : d_light;
            double ll = norm3(lsrc);
            double lh[3] = {lsrc[0] / ll, lsrc[1] / ll, lsrc[2] / ll};
            double ld = dot3(lh, dl);
            for (int c = 0; c < 3; ++c) dst[c] += (dl[c] - lh[c] * ld) / ll;
        }
        {
            double nd = dot3(f.nn, dnn);
            for (int c = 0; c < 3; ++c) d_normal[3 * g + c] += (dnn[c] - f.nn[c] * nd) / f.nlen;
        }
        {
            double vd = dot3(f.vdir, dv);
            for (int c = 0; c < 3; ++c) dmu[c] -= (dv[c] - f.vdir[c] * vd) / f.vlen;
        }
        }
    opacity:
        /* ---- opacity ---- */
        d_opacity_logit[g] += g_opacity[g] * me[3] * f.sig_o * (1.0 - f.sig_o);
        dme[3] += g_opacity[g] * f.sig_o;
        /* ---- conic -> Sigma' ---- */
        double A = f.cov[0], B = f.cov[1], Cc = f.cov[2], D2 = f.det * f.det;
        const double* gc = g_conic + 3 * g;
        double dA = (gc[0] * (-Cc * Cc) + gc[1] * (B * Cc) + gc[2] * (-B * B)) / D2;
        double dB = (gc[0] * (2.0 * B * Cc) + gc[1] * (-(A * Cc + B * B)) + gc[2] * (2.0 * A * B)) / D2;
        double dC = (gc[0] * (-B * B) + gc[1] * (A * B) + gc[2] * (-A * A)) / D2;
        double G2[4] = {dA, 0.5 * dB, 0.5 * dB, dC};
        /* Sigma' = T Sigma T^T: dSigma = T^T G2 T, dT = 2 G2 T Sigma */
        double dSig[9], dT[6], dJ[6];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b) s += f.T[3 * a + i] * G2[2 * a + b] * f.T[3 * b + j];
                dSig[3 * i + j] = s;
            }
        for (int a = 0; a < 2; ++a)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int b = 0; b < 2; ++b)
                    for (int k = 0; k < 3; ++k) s += G2[2 * a + b] * f.T[3 * b + k] * f.Sig[3 * k + j];
                dT[3 * a + j] = 2.0 * s;
            }
        /* T = J W  ->  dJ = dT W^T */
        for (int a = 0; a < 2; ++a)
            for (int k = 0; k < 3; ++k) {
                double s = 0.0;
                for (int j = 0; j < 3; ++j) s += dT[3 * a + j] * R[3 * k + j];
                dJ[3 * a + k] = s;
            }
        double x = f.mc[0], y = f.mc[1], z = f.mc[2];
        double fx = cam->fx, fy = cam->fy;
        double dmc[3] = {0, 0, 0};
        /* J00 = fx/z, J02 = -fx txc/z, J11 = fy/z, J12 = -fy tyc/z */
        dmc[2] += dJ[0] * (-fx / (z * z)) + dJ[4] * (-fy / (z * z));
        if (f.clampx) {
            dmc[2] += dJ[2] * (fx * f.txc / (z * z));
        } else {
            dmc[0] += dJ[2] * (-fx / (z * z));
            dmc[2] += dJ[2] * (2.0 * fx * x / (z * z * z));
        }
        if (f.clampy) {
            dmc[2] += dJ[5] * (fy * f.tyc / (z * z));
        } else {
            dmc[1] += dJ[5] * (-fy / (z * z));
            dmc[2] += dJ[5] * (2.0 * fy * y / (z * z * z));
        }
        /* mean2D: u = fx x/z + cx, v = fy y/z + cy */
        const double* gu = g_uv + 2 * g;
        dmc[0] += gu[0] * fx / z;
        dmc[1] += gu[1] * fy / z;
        dmc[2] += -gu[0] * fx * x / (z * z) - gu[1] * fy * y / (z * z);
        for (int j = 0; j < 3; ++j) dmu[j] += R[j] * dmc[0] + R[3 + j] * dmc[1] + R[6 + j] * dmc[2];
        for (int j = 0; j < 3; ++j) d_mean[3 * g + j] += dmu[j];
        /* Sigma = M M^T, M = R_q S  ->  dM = 2 dSigma M */
        double dM[9];
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) {
                double s = 0.0;
                for (int j = 0; j < 3; ++j) s += dSig[3 * i + j] * f.M[3 * j + k];
                dM[3 * i + k] = 2.0 * s;
            }
        double dR[9];
        for (int k = 0; k < 3; ++k) {
            double ds = 0.0;
            for (int i = 0; i < 3; ++i) {
                ds += f.Rq[3 * i + k] * dM[3 * i + k];
                dR[3 * i + k] = dM[3 * i + k] * f.S[k];
            }
            d_log_scale[3 * g + k] += ds * f.S[k];
        }
        double jac[4][9], dqn[4];
        quat_rot_jac(f.qn, jac);
        for (int k = 0; k < 4; ++k) {
            double s = 0.0;
            for (int i = 0; i < 9; ++i) s += jac[k][i] * dR[i];
            dqn[k] = s;
        }
        const double* q = quat + 4 * g;
        double ql = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        double qd = f.qn[0] * dqn[0] + f.qn[1] * dqn[1] + f.qn[2] * dqn[2] + f.qn[3] * dqn[3];
        for (int k = 0; k < 4; ++k) d_quat[4 * g + k] += (dqn[k] - f.qn[k] * qd) / ql;
    }
}

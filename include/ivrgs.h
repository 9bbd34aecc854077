/*
 * ivrgs.h -- C ABI of libivrgs.so, the GB300 (sm_103a) rasterizer for composed, editable
 * 3D Gaussians (iVR-GS, arXiv 2504.17954).
 *
 * The path: compose basic models and apply edits (Sec. 4.5, 4.6) -> project each Gaussian
 * to the image and shade it with Blinn-Phong (Sec. 3, Sec. 4.3) -> bin the projected
 * footprints into screen tiles and radix-sort them by (tile, depth) -> composite every
 * pixel front to back (Sec. 3, second equation) -> and the reverse mode of all of it.
 *
 * Conventions shared by every entry point
 *   - Every pointer named d_* and every pointer inside the structs below is DEVICE memory
 *     owned by the caller. The library never allocates or frees device memory; where it
 *     needs scratch space it takes a caller-provided workspace whose size a *_workspace
 *     query returns.
 *   - Host structs and host arrays (cameras, edits, bg) are read during the call only.
 *   - `stream` is a cudaStream_t (0 = legacy default stream). Every call is asynchronous on
 *     that stream and does not synchronise, except ivrgs_bin in IVRGS_BIN_EXACT mode, which
 *     reads the pair count back to the host.
 *   - Return value: IVRGS_OK or an error code; no exception crosses the ABI.
 *     ivrgs_last_error() returns a message for the calling thread's last failure.
 *   - Argument errors are detected on the host before anything is launched.
 *   - Layouts are structure-of-arrays, float32 unless stated, row-major, no padding
 *     between elements. Alignment: 16 bytes for float4-typed arrays (conic_o, rgbd,
 *     quat, kads), 8 bytes for xy and keys, 4 bytes otherwise.
 *
 * Camera model: world -> camera x_c = R x + t (camera looks along +z, x right, y down),
 * pixel (i, j) is sampled at (i + 0.5, j + 0.5), u = fx x_c/z_c + cx, v = fy y_c/z_c + cy.
 * Images of all views are packed in one buffer: view v occupies pixels
 * [pix_offset, pix_offset + W*H), row-major.
 *
 * Parameters fixed by the 3DGS lineage the paper builds on (the paper itself is silent):
 * opacity = sigmoid(logit), scale = exp(log s), Sigma' dilated by `lowpass` * I, x/z and
 * y/z clamped to 1.3x the half field of view inside the Jacobian, Gaussians at z <= znear
 * culled, radius = ceil(3 sqrt(lambda_max(Sigma'))), alpha = min(0.99, o' G), alpha < 1/255
 * skipped, the walk ends before a Gaussian that would take the transmittance below 1e-4.
 */
#ifndef IVRGS_H
#define IVRGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ivrgs_status;
enum {
    IVRGS_OK = 0,
    IVRGS_ERR_INVALID_ARG = 1, /* bad pointer, size, alignment or enum */
    IVRGS_ERR_CAPACITY = 2,    /* output/workspace too small; the required size is reported */
    IVRGS_ERR_CUDA = 3,        /* a CUDA runtime call or launch failed */
    IVRGS_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up (see ivrgs_bin) */
    IVRGS_ERR_UNSUPPORTED = 5  /* valid request this library version does not implement */
};

#define IVRGS_MAX_VIEWS 128    /* views per call (cameras travel as kernel parameters) */
#define IVRGS_MAX_MODELS 1024  /* basic models per composed scene */
#define IVRGS_EDIT_STRIDE 8    /* floats per model in the edit table */
#define IVRGS_MAX_PAIRS ((int64_t)1 << 30) /* (tile, Gaussian) pairs per ivrgs_bin call */

enum { IVRGS_FP32 = 0, IVRGS_MIXED = 1, IVRGS_VQ = 2 };
#define IVRGS_VQ_ATTRS 8       /* codebooks per model: log_scale, quat, opacity_logit, dcolor, k_a, k_d, k_s, beta */
#define IVRGS_VQ_MAX_K 256     /* codebook entries at most (u8 indices) */
#define IVRGS_ANCHOR_CHUNK 256 /* Gaussians per float32 position anchor in IVRGS_MIXED storage */
enum { IVRGS_BIN_EXACT = 0, IVRGS_BIN_CAPACITY = 1, IVRGS_BIN_CULL = 2 };

/* One pinhole view. light_dir is the direction towards an orbital (directional) light in
   world space, used when headlight == 0; with headlight != 0 the light sits at the camera
   and l equals the viewing direction v of each Gaussian (Sec. 3, Blinn-Phong paragraph). */
typedef struct {
    int32_t W, H;
    float fx, fy, cx, cy;
    float R[9];        /* world -> camera rotation, row-major */
    float t[3];
    float campos[3];   /* camera centre in world space (= -R^T t) */
    float znear;
    int32_t headlight;
    float light_dir[3];
    int64_t pix_offset;
} ivrgs_camera;

/* Per-basic-model edits (Sec. 4.5): palette colour c_p replaces the model's colour
   anchor, the opacity of all its Gaussians is multiplied by opacity_scale, and a model with
   visible == 0 is left out of the composition. */
typedef struct {
    float palette[3];
    float opacity_scale;
    int32_t visible;
} ivrgs_model_edit;

/* Global light edits (Sec. 4.5, Sec. 4.6): magnitude k' = lambda * k + bias for
   k = (k_a, k_d, k_s, beta); with dir_on != 0 the direction dir (any non-zero length; dir / |dir|
   is used) replaces the light_dir of every view that has an orbital light (Sec. 4.6 learns one
   light direction for the composed model). */
typedef struct {
    float lambda[4];
    float bias[4];
    float dir[3];
    int32_t dir_on;
} ivrgs_light;

/* Editable Gaussians (Sec. 4.3 attribute set), structure of arrays, n entries.
   precision IVRGS_FP32: float32 arrays mean [n][3], log_scale [n][3], quat [n][4] as
   (w, x, y, z) (need not be normalised), opacity_logit [n], dcolor [n][3] (offset colour dc,
   c_v = c_p + dc), normal [n][3] (need not be normalised), kads [n][4] = (k_a, k_d, k_s,
   beta); anchor unused.
   precision IVRGS_MIXED (16-bit storage, float32 arithmetic): mean FP16 [n][3] offsets, with
   the stored mean defined as the float32 sum anchor[g / IVRGS_ANCHOR_CHUNK] + offset
   (anchor: float32 [ceil(n / 256)][3]); log_scale BF16 [n][3]; quat FP16 [n][4]; opacity_logit
   FP16 [n]; dcolor BF16 [n][3]; normal BF16 [n][3]; kads FP16 [n][4]. ivrgs_pack_mixed
   writes this layout.
   precision IVRGS_VQ (Sec. 4.4: vector quantisation; mean and normal exact, every other
   attribute an index into a scalar codebook shared by all components of that attribute
   within one basic model): mean and normal float32 as in IVRGS_FP32; uint8 indices
   log_scale [n][3], quat [n][4], opacity_logit [n], dcolor [n][3], kads [n][4]; codebook
   float32 [n_models][IVRGS_VQ_ATTRS][vq_k], the attributes in the order log_scale, quat,
   opacity_logit, dcolor, k_a, k_d, k_s, beta (kads component j uses codebook 4 + j).
   ivrgs_vq_build writes this layout.
   model_id [n] (basic model of each Gaussian, < n_models) in all. Gradients are always
   float32 with the FP32 layout (w.r.t. the decoded values for IVRGS_MIXED and IVRGS_VQ). */
typedef struct {
    int64_t n;
    int32_t precision; /* IVRGS_FP32, IVRGS_MIXED or IVRGS_VQ */
    int32_t n_models;
    void* mean;
    void* log_scale;
    void* quat;
    void* opacity_logit;
    void* dcolor;
    void* normal;
    void* kads;
    uint16_t* model_id;
    float* anchor;   /* IVRGS_MIXED: float32 [ceil(n / 256)][3]; unused otherwise */
    float* codebook; /* IVRGS_VQ: float32 [n_models][IVRGS_VQ_ATTRS][vq_k]; unused otherwise */
    int32_t vq_k;    /* IVRGS_VQ: codebook entries, 1..IVRGS_VQ_MAX_K */
    /* Optional 3DGS colour (the view-dependent SH colour of Sec. 3 / Sec. 4.2, any storage):
       float32 [n][(sh_degree + 1)^2][3] coefficients, sh_degree 0..3. If sh != NULL the colour
       is max(0, sum_k sh_k Y_k(d) + 0.5) with d = (mean - campos) / |mean - campos| and the real
       SH basis Y_k (orthonormal, Condon-Shortley sign) instead of the Blinn-Phong shading; dcolor,
       normal, kads and the palette, lambda, b and light edits then do not enter; the opacity and
       visibility edits do. In a gradient struct, sh (same layout) receives dL/dsh. */
    float* sh;
    int32_t sh_degree;
} ivrgs_gaussians;

/* Projected Gaussians, one record per (view v, Gaussian g) at index v * n + g.
   xy [.][2] = (u, v) pixel-space mean; conic_o [.][4] = (g, b, c, o') with K = (a, b; b, c) the
   inverse of Sigma', g = a - b^2 / c = 1 / Sigma'_xx (K in completed-square form: the exponent
   -(a e_x^2 + 2 b e_x e_y + c e_y^2) / 2 is evaluated as -(c (e_y + (b/c) e_x)^2 + g e_x^2) / 2,
   which keeps its float32 rounding small for long, thin Gaussians) and o' the edited opacity;
   rgbd [.][4] = (r, g, b, depth) shaded colour
   and camera-space depth; radius [.] = ceil(3 sqrt(lambda_max)) in pixels, 0 if culled
   (the other fields of a culled record are unspecified). */
typedef struct {
    int64_t n;
    int32_t n_views;
    float* xy;
    float* conic_o;
    float* rgbd;
    int32_t* radius;
} ivrgs_projected;

/* Tile bins. Global tile ids run over all views: view v's tiles start at the sum of the
   tile counts of views < v, row-major inside a view. The pairs (tile, Gaussian) are ordered
   by (tile, bits of the float depth), ties in (view, Gaussian) order -- i.e. ascending in the
   64-bit key (tile << 32) | bits(depth). tiles [capacity] = global tile id of each sorted pair;
   values [capacity] = Gaussian index g of each sorted pair; ranges [n_tiles][2] = [start, end)
   of each tile's run ((0, 0) for an empty tile). d_n_pairs: device uint64 scalar receiving the
   number of pairs (in CAPACITY mode a value > capacity means the outputs are incomplete). */
typedef struct {
    int32_t tile_w, tile_h; /* tile_w = 16; tile_h = 16 or 8 (other shapes: IVRGS_ERR_UNSUPPORTED) */
    int64_t n_tiles;
    int64_t capacity;
    uint32_t* tiles;
    uint32_t* values;
    uint32_t* ranges;
    uint64_t* d_n_pairs;
    int64_t n_pairs; /* out: filled by IVRGS_BIN_EXACT mode */
} ivrgs_bins;

/* Message of the calling thread's last failed call ("" if none). Never NULL. */
const char* ivrgs_last_error(void);

/* Library version (major * 10000 + minor * 100 + patch). */
int32_t ivrgs_version(void);

/* Launch-shape options (process-wide; measurement-driven tuning, the paper has no counterpart):
   "render_pixels_per_thread" and "render_bwd_pixels_per_thread" (1, 2, 4 or 8, or 0 = by tile
   count, the default: 4 from 3072 tiles per call, else 1): pixels each thread
   of the forward / backward blend owns; "sort_match" (0 or 1): rank radix digits with warp
   ballots (0) or match.any (1); "sort_scan" (0 or 1): radix-pass offsets by decoupled
   look-back (0, one kernel per pass) or reduce-then-scan (1: a histogram kernel, a per-digit
   scan and the scatter; no device-side waits); "sort_early" (0 or 1): in the tile-id passes, a
   look-back radix tile publishes its digit counts after (0) or before (1) ranking its keys (the
   depth passes always publish before); "render_split" (0 to 4): both blends walk every tile's
   run with one CTA (2), or cut runs longer than "render_split_min" entries (32, 64, 128,
   256 (default), 384, 512, 768, 1024, 2048 or 4096) into up to 8 chunks walked by the 8 CTAs of a
   thread-block cluster whose partial results merge through distributed shared memory (1), or
   do so when the call has fewer than 304 tiles (0, the default: two tiles per SM, below which
   the heaviest tiles' serial walks are the whole launch), or do so in the backward only, below
   304 tiles (3), or walk the runs longer than render_split_min unsplit in a launch of their
   own, started first, below 304 tiles (4). The kernel of the long runs runs on a library-owned stream beside the
   kernel of the other tiles (forked from and joined back to the caller's stream, capturable).
   Results are identical for
   every setting, except that the split walk regroups the float32 transmittance products (last
   bits; a termination decision only at a float32 near-tie).
   Returns IVRGS_ERR_INVALID_ARG for an unknown name or value. */
ivrgs_status ivrgs_set_option(const char* name, int64_t value);
ivrgs_status ivrgs_get_option(const char* name, int64_t* value);

/* Number of floats in an edit table for n_models models: IVRGS_EDIT_STRIDE * n_models + 12.
   Layout: per model m, [c_p(3), opacity scale, visible (0/1), 0, 0, 0]; then lambda(4), b(4),
   global light (dir(3), on (0/1)). The edit-gradient buffer of ivrgs_render_backward has the
   same layout (the global light's slots receive d dir while it is on) followed by 4 floats per
   view (d light_dir (3), 0; zero for views whose light the global one replaces). */
int64_t ivrgs_edit_table_floats(int32_t n_models);

/* Composition and edits (Sec. 4.5: the composed model is the concatenation of the basic
   models' Gaussian attributes; colour, opacity and light edits; Sec. 4.6: lambda, b).
   models: host array of n_models structs, each naming one basic model's device arrays
   (their model_id and n_models fields are ignored). If `composed` is non-NULL its arrays
   (composed->n must equal the sum of the models' n) receive the concatenation in model
   order and model_id is set to the model index. If `composed` is NULL only the edit table is
   written, so re-editing costs O(n_models). d_edit_table: device float array of
   ivrgs_edit_table_floats(n_models) entries, written from `edits` and `light`. */
ivrgs_status ivrgs_compose_edit(const ivrgs_gaussians* models, int32_t n_models, const ivrgs_model_edit* edits,
                                const ivrgs_light* light, ivrgs_gaussians* composed, float* d_edit_table,
                                void* stream);

/* EWA projection + Blinn-Phong shading with edits applied (Sec. 3 first equation and
   the Blinn-Phong system; Sec. 4.3 c_v = c_p + dc; Sec. 4.5/4.6 edits). For every view
   v < n_views and Gaussian g: culls hidden models, z_c <= znear and det(Sigma') <= 0;
   Sigma = R(q) diag(exp 2 s) R(q)^T, Sigma' = J R Sigma R^T J^T + lowpass I; writes
   out (n = g->n, n_views). The depth (sort key, near-plane test) is the float32 chain
   fma(R22, mz, fma(R21, my, fma(R20, mx, t2))), each step one correctly rounded fused
   multiply-add, so sort keys are exactly reproducible. */
ivrgs_status ivrgs_project(const ivrgs_gaussians* g, const float* d_edit_table, const ivrgs_camera* cams,
                           int32_t n_views, float lowpass, ivrgs_projected* out, void* stream);

/* Workspace bytes ivrgs_bin needs for p->n * n_views records (below IVRGS_MAX_PAIRS, i.e. 2^30, as
   for the pairs: the radix look-back carries 30-bit counts) and `capacity` pairs
   (about 57 bytes per record plus 9 per pair). Tiles are tile_w = 16 pixels wide and tile_h = 16
   or 8 high (any other shape: IVRGS_ERR_UNSUPPORTED); the tile shape is not the paper's (it does
   not fix one), a launch shape picked for speed, and it decides the tile lists (a Gaussian is
   listed for every tile of its rectangle) and so, at pixels outside its 3-sigma radius but
   inside its rectangle, the image. */
ivrgs_status ivrgs_bin_workspace(int64_t n, int32_t n_views, const ivrgs_camera* cams, int32_t tile_w,
                                 int32_t tile_h, int64_t capacity, size_t* bytes);

/* Tile binning by radix sort (the tile-based rasterisation of 3DGS that Sec. 3 builds on:
   projected Gaussians are composited in depth order per screen tile). Per record: tile
   rectangle (half-open) x0 = clamp(floor((u - r)/tile_w), 0, Gx),
   x1 = clamp(floor((u + r)/tile_w) + 1, 0, Gx) (the same for y with tile_h) evaluated in
   float32; one pair per covered tile. out->tile_w and out->tile_h give the tile shape (16 x 16
   or 16 x 8); every later call with these bins uses it. Ordering: the covered records are radix-sorted by the bits of their float
   depth (stable, 4 passes of 8 bits), their pairs are emitted in that order and then
   radix-sorted by tile id (stable, one pass per 8 bits of the largest tile id); both sorts
   are onesweep LSD sorts with decoupled look-back. The result equals the stable sort of all
   pairs by (tile << 32 | depth bits).
   mode IVRGS_BIN_EXACT: counts the pairs, copies the count to the host (synchronises the
   stream), returns IVRGS_ERR_CAPACITY with out->n_pairs = required count if it exceeds
   out->capacity, else finishes and sets out->n_pairs.
   mode IVRGS_BIN_CAPACITY: never synchronises (usable inside CUDA graph capture); works
   on min(count, capacity) pairs and leaves the true count in *out->d_n_pairs.
   mode | IVRGS_BIN_CULL (no counterpart in the paper; a refinement that leaves every
   composited value unchanged): a pair is emitted only if its tile meets the Gaussian's
   opacity cut-off ellipse, q(e) = a e_x^2 + 2 b e_x e_y + c e_y^2 <= 2 ln(255 o') + 0.25 for
   some point e of the box spanned by the tile's pixel centres (conic (a, b, c) and o' from
   p->conic_o, a = g + b^2 / c). Outside that
   ellipse alpha < 1/255, so the compositing skips the Gaussian at every pixel of a dropped
   tile. The lists are the rectangle lists above with those pairs removed, in the same order.
   Conics with a c > 4096 (a c - b^2) keep their whole rectangle.
   A device-side wait of the sort that exceeds its iteration bound sets a flag in the
   workspace; EXACT mode reports it as IVRGS_ERR_TIMEOUT, CAPACITY mode via
   ivrgs_bin_check(). An emission that disagrees with the count pass (never expected) is
   reported the same way as IVRGS_ERR_CUDA. */
ivrgs_status ivrgs_bin(const ivrgs_projected* p, const ivrgs_camera* cams, int32_t n_views, int32_t mode,
                       void* d_workspace, size_t ws_bytes, ivrgs_bins* out, void* stream);

/* Reads (synchronously) the error flag a previous ivrgs_bin left in d_workspace:
   IVRGS_OK, IVRGS_ERR_TIMEOUT or IVRGS_ERR_CUDA (see ivrgs_bin). */
ivrgs_status ivrgs_bin_check(const void* d_workspace, void* stream);

/* Front-to-back alpha compositing per tile (Sec. 3 second equation, C = sum T_i alpha_i c_i,
   T_i = prod_{j<i}(1 - alpha_j); alpha channel as in Sec. 4.2). One CTA per tile (16 x 16 or
   16 x 8, from b->tile_h).
   Outputs per packed pixel: d_rgba [.][4] = (C + T bg, 1 - T), d_final_T [.] = T after the
   last contributor, d_last [.] = 1 + position (within the tile's run) of the last
   contributing Gaussian, 0 if none. bg: host float[3]. */
ivrgs_status ivrgs_render(const ivrgs_projected* p, const ivrgs_bins* b, const ivrgs_camera* cams,
                          int32_t n_views, const float* bg, float* d_rgba, float* d_final_T, uint32_t* d_last,
                          void* stream);

/* Auxiliary maps with the compositing weights of ivrgs_render (Sec. 4.2 first equation: depth
   and normal maps D, N = sum_i T_i alpha_i {d_i, n_i}; Sec. 4.3: offset-colour and coefficient
   maps sum_i T_i alpha_i {dc_i, k_i}; the attribute render modes of Sec. 4.7). Inputs: the
   Gaussians g and edit table of the projection that produced p, and the bins b. Output per
   packed pixel, d_aux [.][12] float (16-byte aligned): depth (camera z), normal (3, world,
   unit per Gaussian), dc (3), k' = lambda k + b (4: k_a, k_d, k_s, beta), 1 - T. The walk takes
   exactly the contributors and weights of ivrgs_render (the last channel equals its alpha).
   No background term. */
ivrgs_status ivrgs_render_aux(const ivrgs_gaussians* g, const float* d_edit_table, const ivrgs_projected* p,
                              const ivrgs_bins* b, const ivrgs_camera* cams, int32_t n_views, float* d_aux,
                              void* stream);

/* Workspace bytes ivrgs_render_aux_backward needs for n Gaussians and n_views views. */
ivrgs_status ivrgs_render_aux_backward_workspace(int64_t n, int32_t n_views, size_t* bytes);

/* Reverse mode of ivrgs_render_aux (Sec. 4.2 first equation: the maps composite each Gaussian's
   values with the weights T_i alpha_i, no background; the last channel is 1 - T). Inputs: the
   same g, d_edit_table, p, b, cams and lowpass as the forward, ivrgs_render's d_final_T and
   d_last, and d_dL_daux [.][12] = dL/d(the 11 channels of ivrgs_render_aux, 1 - T) per packed
   pixel (16-byte aligned). The walk is the colour reverse mode's with the values in place of the
   colour. Outputs (overwritten): grad arrays with the layout of g (float32, model_id unused) =
   dL/d{mean, log_scale, quat, opacity_logit, dcolor, normal, kads} (SH coefficients, if g has
   them, receive zero: the maps do not depend on the colour); d_edit_grad
   (ivrgs_edit_table_floats(n_models) + 4 * n_views floats) = dL/d{opacity scale} per model and
   dL/d{lambda, b} (palette colours and lights: zero). d_workspace: at least
   ivrgs_render_aux_backward_workspace bytes, 256-byte aligned (IVRGS_ERR_CAPACITY if smaller). */
ivrgs_status ivrgs_render_aux_backward(const ivrgs_gaussians* g, const float* d_edit_table,
                                       const ivrgs_projected* p, const ivrgs_bins* b, const ivrgs_camera* cams,
                                       int32_t n_views, float lowpass, const float* d_final_T,
                                       const uint32_t* d_last, const float* d_dL_daux, void* d_workspace,
                                       size_t ws_bytes, ivrgs_gaussians* grad, float* d_edit_grad, void* stream);

/* Workspace bytes ivrgs_render_backward needs for n Gaussians and n_views views. */
ivrgs_status ivrgs_render_backward_workspace(int64_t n, int32_t n_views, size_t* bytes);

/* Reverse mode of ivrgs_compose_edit (edit table) + ivrgs_project + ivrgs_render.
   Inputs: the same g, d_edit_table, p, b, cams, lowpass and bg as the forward, its
   d_final_T and d_last, and d_dL_drgba [.][4] = dL/d(r, g, b, alpha) per packed pixel.
   The blend is walked back to front from each pixel's last contributor with the
   transmittance recomputed as T_i = T_{i+1} / (1 - alpha_i) from the stored final T.
   Outputs (overwritten): grad arrays with the layout of g (float32, model_id unused) =
   dL/d{mean, log_scale, quat, opacity_logit, dcolor, normal, kads}; d_edit_grad
   (ivrgs_edit_table_floats(n_models) + 4 * n_views floats) = dL/d{c_p, opacity scale} per
   model, dL/d{lambda, b}, and dL/d light_dir per view (zero for headlight views).
   The workspace also holds, on return, the per-(view, Gaussian) gradients of the 2D
   quantities: float4 [V*n] (du, dv, da, db), float4 [V*n] (dc, do', dr, dg), float [V*n] (db). */
ivrgs_status ivrgs_render_backward(const ivrgs_gaussians* g, const float* d_edit_table, const ivrgs_projected* p,
                                   const ivrgs_bins* b, const ivrgs_camera* cams, int32_t n_views, float lowpass,
                                   const float* bg, const float* d_final_T, const uint32_t* d_last,
                                   const float* d_dL_drgba, void* d_workspace, size_t ws_bytes,
                                   ivrgs_gaussians* grad, float* d_edit_grad, void* stream);

/* Spatial ordering keys for packing (precision pattern; a storage-layout helper with no
   counterpart in the paper): d_keys[g] = (model_id[g] << 30) | Morton code (10 bits per axis)
   of mean[g] quantised inside the box [lo, hi] (host float[3] each). Sorting the keys
   (stable, any sort) and passing the permutation to ivrgs_pack_mixed keeps each model
   contiguous and makes every 256-Gaussian chunk spatially compact, so the FP16 offsets from
   its anchor are small. g must be IVRGS_FP32. */
ivrgs_status ivrgs_morton_keys(const ivrgs_gaussians* g, const float* lo, const float* hi, uint64_t* d_keys,
                               void* stream);

/* Packs float32 Gaussians into IVRGS_MIXED storage (Sec. 4.3 attributes, 16-bit floats,
   round to nearest): out[k] = in[d_order[k]] (d_order: device uint32 [n], a permutation; NULL
   for the identity). Each chunk of 256 output Gaussians gets the float32 anchor at the centre
   of its means' bounding box and FP16 offsets from it. out->n must equal in->n; out's arrays
   are caller-owned with the IVRGS_MIXED layout, out->anchor included. */
ivrgs_status ivrgs_pack_mixed(const ivrgs_gaussians* in, const uint32_t* d_order, ivrgs_gaussians* out,
                              void* stream);

/* ivrgs_render_backward that ADDS its gradients to grad and to the first
   ivrgs_edit_table_floats(n_models) floats of d_edit_grad (the per-view light gradients of
   this call's cameras, which follow, are overwritten) instead of overwriting them: the
   backward of a set of views rendered in several calls (view waves, when one call would
   exceed IVRGS_MAX_PAIRS pairs or IVRGS_MAX_VIEWS views) is the sum of the calls' backwards
   (Sec. 3 Eq. C is per pixel; the views share only the Gaussians). Same arguments otherwise. */
ivrgs_status ivrgs_render_backward_accumulate(const ivrgs_gaussians* g, const float* d_edit_table,
                                              const ivrgs_projected* p, const ivrgs_bins* b, const ivrgs_camera* cams,
                                              int32_t n_views, float lowpass, const float* bg, const float* d_final_T,
                                              const uint32_t* d_last, const float* d_dL_drgba, void* d_workspace,
                                              size_t ws_bytes, ivrgs_gaussians* grad, float* d_edit_grad,
                                              void* stream);

/* Bytes of the device array that ivrgs_render_backward_static uses as its scratch. */
#define IVRGS_STATIC_SCRATCH_BYTES ((size_t)32 << 20)

/* ivrgs_render_backward without a workspace argument. The paper has no counterpart: this
   entry point exists for callers that cannot call cudaMalloc, for example a plugin running
   inside a host visualisation application that owns all device memory, or an interactive
   editing loop that must not stall on the device-wide synchronisation an allocation can
   cause. Its scratch is one array of IVRGS_STATIC_SCRATCH_BYTES bytes compiled into the
   library; every GPU that loads the library holds it until the process exits.
   Arguments, outputs and semantics are those of ivrgs_render_backward minus d_workspace and
   ws_bytes; the caller still provides every input and output array. The call allocates
   nothing (no cudaMalloc, cudaFree or allocating library routine).
   Limit: the workspace ivrgs_render_backward_workspace(n, n_views) reports (36 bytes per
   view-Gaussian record plus 256) must fit, i.e. n * n_views <= 932,060; a larger request
   returns IVRGS_ERR_CAPACITY before anything is launched.
   The first call on a device looks up the array's device address with that device current
   and caches it with the current CUDA context, so make that first call before any stream
   capture; a call under a different context (after cudaDeviceReset, say) looks the address
   up again, and that call too belongs before any capture. Every call uses the
   same array and leaves its contents behind (each call clears what must start at zero);
   calls that overlap on the GPU -- concurrent streams, host threads or processes sharing
   the context -- race on the array, so the caller must serialise them. */
ivrgs_status ivrgs_render_backward_static(const ivrgs_gaussians* g, const float* d_edit_table,
                                          const ivrgs_projected* p, const ivrgs_bins* b, const ivrgs_camera* cams,
                                          int32_t n_views, float lowpass, const float* bg, const float* d_final_T,
                                          const uint32_t* d_last, const float* d_dL_drgba, ivrgs_gaussians* grad,
                                          float* d_edit_grad, void* stream);

/* ---------------------------------------------------------------------------------------
   Inverse volume exploration (Sec. 4.6): all Gaussian attributes stay fixed; the per-model
   palette colour c_p and opacity scale, the global lambda and b, and (orbital light) the global
   light direction as polar and azimuthal angles are fitted to a reference image by gradient
   steps on a combined L1 / SSIM loss (Sec. 5: learning rate 0.01, 1000 iterations).
   --------------------------------------------------------------------------------------- */
enum {
    IVRGS_LEARN_COLOR = 1,           /* c_p of every model */
    IVRGS_LEARN_OPACITY = 2,         /* opacity scale of every model */
    IVRGS_LEARN_LIGHT_MAGNITUDE = 4, /* lambda and b */
    IVRGS_LEARN_LIGHT_DIRECTION = 8  /* polar / azimuth of the edit table's global light (if on) */
};

/* Workspace bytes of ivrgs_image_loss for these views. */
ivrgs_status ivrgs_image_loss_workspace(const ivrgs_camera* cams, int32_t n_views, size_t* bytes);

/* Image loss of a rendering against a reference (the 3DGS loss that the paper's combination of
   L1 and SSIM denotes): loss = (1 - lambda_ssim) L1 + lambda_ssim (1 - SSIM) over the R, G, B
   channels of all views, L1 = mean |x - y|, SSIM = mean of the per-pixel, per-channel structural
   similarity with an 11 x 11 Gaussian window (sigma 1.5, normalised), C1 = 0.01^2, C2 = 0.03^2,
   zero padding at each view's border. d_rgba, d_target: packed images [.][4] (alpha ignored),
   16-byte aligned. Writes d_loss[0..2] = (loss, L1, SSIM) and d_dL_drgba [.][4] = dloss/d(r, g,
   b) with 0 for alpha, for the views' pixels only. With lambda_ssim = 0 (the plain L1 loss) the
   SSIM passes are skipped and d_loss[2] is written as 0. Workspace: ivrgs_image_loss_workspace
   bytes, 256-byte aligned. */
ivrgs_status ivrgs_image_loss(const float* d_rgba, const float* d_target, const ivrgs_camera* cams, int32_t n_views,
                              float lambda_ssim, void* d_workspace, size_t ws_bytes, float* d_loss,
                              float* d_dL_drgba, void* stream);

/* Floats of the optimiser state for n_models models: 2 (4 n_models + 10) + 3 = first and second
   moments of every learnable value, the light's (polar, azimuth) angles and the step count. */
int64_t ivrgs_edit_adam_state_floats(int32_t n_models);

/* Sets the moments and the step count to zero and the angles to those of the edit table's
   global light (polar from +z, azimuth from +x). */
ivrgs_status ivrgs_edit_adam_init(const float* d_edit_table, int32_t n_models, float* d_state, void* stream);

/* One Adam step (Kingma and Ba; bias-corrected moments, step = lr m^ / (sqrt(v^) + eps)) on the
   edit-table values selected by `learn` (IVRGS_LEARN_*), with d_edit_grad laid out as the
   edit-gradient buffer of ivrgs_render_backward. The light direction is stepped through its
   angles and written back to the table as a unit vector (only while the global light is on).
   The step count lives in d_state, so a captured CUDA graph can replay whole iterations. */
ivrgs_status ivrgs_edit_adam(float* d_edit_table, const float* d_edit_grad, int32_t n_models, float* d_state,
                             int32_t learn, float lr, float beta1, float beta2, float eps, void* stream);

/* ---------------------------------------------------------------------------------------
   Vector quantisation (Sec. 4.4): codebooks by k-means per basic model and attribute (all
   attributes but the mean and the normal; one scalar codebook per attribute shared by its
   components), one uint8 index per component.
   --------------------------------------------------------------------------------------- */
/* Workspace bytes of ivrgs_vq_build. */
ivrgs_status ivrgs_vq_build_workspace(int32_t n_models, int32_t k, size_t* bytes);

/* Builds the IVRGS_VQ storage of src (IVRGS_FP32 with model_id): for every (model, attribute)
   k centroids initialised evenly over [min, max] of its values, then `iters` Lloyd iterations
   (nearest centroid by midpoints of the sorted centroids, a value on a midpoint to the lower
   one; each centroid moved to the mean of its values, an empty one kept; order kept by a
   running maximum); then every component's index of its nearest centroid. Writes out's index
   arrays and codebook ([n_models][IVRGS_VQ_ATTRS][k]); out->mean, normal and model_id are not
   touched (they may share src's arrays). out: precision IVRGS_VQ, same n and n_models, vq_k = k.
   Workspace 256-byte aligned, ivrgs_vq_build_workspace bytes. */
ivrgs_status ivrgs_vq_build(const ivrgs_gaussians* src, int32_t k, int32_t iters, ivrgs_gaussians* out,
                            void* d_workspace, size_t ws_bytes, void* stream);

/* Opt-in per-kernel timing (measurement support; the paper has no counterpart). With
   on != 0 every kernel launch of the library is bracketed by two CUDA events on its stream.
   Must be off while a stream is being captured into a CUDA graph. */
void ivrgs_prof_enable(int32_t on);

/* Synchronises on the recorded events and returns the length of a report with one line
   "kernel launches total_ms" per kernel launched since the last delivered report. If buf
   holds more than that many bytes (len > length) the report is copied there, NUL-terminated,
   and the totals are reset; otherwise nothing is copied and the totals are kept. */
int64_t ivrgs_prof_report(char* buf, int64_t len);

#ifdef __cplusplus
}
#endif

#endif /* IVRGS_H */

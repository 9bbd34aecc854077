"""FP64 CPU oracle of the editable-Gaussian rasterizer (test infrastructure).

TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the benchmark's CPU-baseline leg
may import this package.  The product (``paper_2504_17954_gb300``) never imports it, and this
package never imports the product.  Inputs come from ``scenegen`` (seeded draws only).

The arithmetic lives in ``ivrgs_oracle.c`` (plain scalar float64 C, see its header for the
passages of the paper each step follows); this module does the bookkeeping:

* composition (Sec. 4.5): the basic models' attributes are concatenated in model order;
* the edit table (Sec. 4.5, 4.6): per model [c_p(3), opacity scale, visible, 0, 0, 0], then
  lambda(4) and b(4), with k' = lambda * (k_a, k_d, k_s, beta) + b, then an optional global
  orbital light direction (l(3), on) that replaces every view's own (Sec. 4.6);
* per view: projection + shading, float32-decided binning, compositing, and the reverse
  mode of all of it.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py`` against closed
forms, invariants, brute force (``oracle/brute.py``) and central finite differences.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ivrgs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libivrgs_oracle.so")
EDIT_STRIDE = 8
# per-pixel decision record: [|ln(255 alpha)|, |ln(T'/1e-4)|, |P|/scale, |ln(oG/0.99)|,
#                             sum of (k+1) over contributors, sum of (k+1)^2 over clamped ones]
N_MARGINS = 6
LOWPASS = 0.3
GUARD = 1.3

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no fast-math, no FP contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrcCamera(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("R", C.c_double * 9), ("t", C.c_double * 3),
                ("campos", C.c_double * 3), ("znear", C.c_double), ("headlight", C.c_int32),
                ("light_dir", C.c_double * 3)]


def _p(a, ct=C.c_double):
    return a.ctypes.data_as(C.POINTER(ct))


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_bin.restype = C.c_int64
    return _lib


# ----------------------------------------------------------------------------------------
@dataclass
class Composed:
    """Concatenated float64 attributes of all basic models (Sec. 4.5)."""
    mean: np.ndarray
    log_scale: np.ndarray
    quat: np.ndarray
    opacity_logit: np.ndarray
    dcolor: np.ndarray
    normal: np.ndarray
    kads: np.ndarray
    model_id: np.ndarray
    n_models: int
    sh: Optional[np.ndarray] = None  # [N, (deg+1)^2, 3]: 3DGS colour instead of Blinn-Phong
    sh_degree: int = -1

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    def arrays(self):
        return [self.mean, self.log_scale, self.quat, self.opacity_logit, self.dcolor, self.normal, self.kads]


PARAMS = ("mean", "log_scale", "quat", "opacity_logit", "dcolor", "normal", "kads")


def compose(models) -> Composed:
    cat = lambda k: np.ascontiguousarray(np.concatenate([np.asarray(getattr(m, k), np.float64) for m in models]))
    mid = np.concatenate([np.full(m.n, i, np.int32) for i, m in enumerate(models)])
    return Composed(*(cat(k) for k in PARAMS), model_id=np.ascontiguousarray(mid), n_models=len(models))


def edit_table(edits) -> np.ndarray:
    M = len(edits.opacity_scale)
    t = np.zeros(M * EDIT_STRIDE + 12, np.float64)
    for m in range(M):
        t[m * EDIT_STRIDE:m * EDIT_STRIDE + 3] = edits.palette[m]
        t[m * EDIT_STRIDE + 3] = edits.opacity_scale[m]
        t[m * EDIT_STRIDE + 4] = 1.0 if edits.visible[m] else 0.0
    t[M * EDIT_STRIDE:M * EDIT_STRIDE + 4] = edits.lam
    t[M * EDIT_STRIDE + 4:M * EDIT_STRIDE + 8] = edits.bias
    ld = getattr(edits, "light_dir", None)
    if ld is not None:  # one light direction for every orbital view (Sec. 4.6)
        t[M * EDIT_STRIDE + 8:M * EDIT_STRIDE + 11] = ld
        t[M * EDIT_STRIDE + 11] = 1.0
    return t


def camera(c) -> OrcCamera:
    oc = OrcCamera()
    oc.W, oc.H = int(c.W), int(c.H)
    oc.fx, oc.fy, oc.cx, oc.cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
    for i in range(9):
        oc.R[i] = float(c.R[i])
    for i in range(3):
        oc.t[i] = float(c.t[i])
        oc.campos[i] = float(c.campos[i])
        oc.light_dir[i] = float(c.light_dir[i])
    oc.znear = float(c.znear)
    oc.headlight = int(c.headlight)
    return oc


# ----------------------------------------------------------------------------------------
@dataclass
class Projected:
    uv: np.ndarray       # [N, 2] float64
    cov: np.ndarray      # [N, 3] Sigma' (A, B, C)
    conic: np.ndarray    # [N, 3] (a, b, c)
    opacity: np.ndarray  # [N]
    rgb: np.ndarray      # [N, 3]
    depth: np.ndarray    # [N]
    radius: np.ndarray   # [N] int32, 0 = culled
    radius_margin: np.ndarray
    # distance of the float64 depth to the nearest float32 rounding midpoint, relative to
    # |t_z| + sum_k |R_zk mu_k| (how far the float32 sort key is from a rounding tie)
    depth_margin: Optional[np.ndarray] = None


def project(comp: Composed, table: np.ndarray, cam, lowpass: float = LOWPASS, guard: float = GUARD) -> Projected:
    n = comp.n
    out = Projected(uv=np.zeros((n, 2)), cov=np.zeros((n, 3)), conic=np.zeros((n, 3)), opacity=np.zeros(n),
                    rgb=np.zeros((n, 3)), depth=np.zeros(n), radius=np.zeros(n, np.int32),
                    radius_margin=np.zeros(n), depth_margin=np.zeros(n))
    oc = camera(cam)
    lib().orc_project(C.c_int64(n), *[_p(a) for a in comp.arrays()], _p(comp.model_id, C.c_int32),
                      *_sh_args(comp), _p(table), C.c_int32(comp.n_models), C.byref(oc), C.c_double(lowpass), C.c_double(guard),
                      _p(out.uv), _p(out.cov), _p(out.conic), _p(out.opacity), _p(out.rgb), _p(out.depth),
                      _p(out.radius, C.c_int32), _p(out.radius_margin), _p(out.depth_margin))
    return out


@dataclass
class Bins:
    keys: np.ndarray      # [P] uint64
    values: np.ndarray    # [P] uint32
    ranges: np.ndarray    # [n_tiles, 2] uint32
    tile_offset: np.ndarray  # [V+1] int64


def bin_pairs(uv32: np.ndarray, radius: np.ndarray, depth32: np.ndarray, sizes: Sequence, tile=(16, 16)) -> Bins:
    """Tile binning + stable ordering from float32 decision inputs ([V, N, 2], [V, N], [V, N])."""
    uv32 = np.ascontiguousarray(uv32, np.float32)
    radius = np.ascontiguousarray(radius, np.int32)
    depth32 = np.ascontiguousarray(depth32, np.float32)
    V, n = radius.shape
    Ws = np.array([s[0] for s in sizes], np.int32)
    Hs = np.array([s[1] for s in sizes], np.int32)
    toff = np.zeros(V + 1, np.int64)
    nt = int(sum(((w + tile[0] - 1) // tile[0]) * ((h + tile[1] - 1) // tile[1]) for w, h in zip(Ws, Hs)))
    ranges = np.zeros((max(nt, 1), 2), np.uint32)
    dummy_k = np.zeros(1, np.uint64)
    dummy_v = np.zeros(1, np.uint32)
    total = lib().orc_bin(C.c_int32(V), C.c_int64(n), _p(uv32, C.c_float), _p(radius, C.c_int32),
                          _p(depth32, C.c_float), _p(Ws, C.c_int32), _p(Hs, C.c_int32), C.c_int32(tile[0]),
                          C.c_int32(tile[1]), _p(dummy_k, C.c_uint64), _p(dummy_v, C.c_uint32), C.c_int64(0),
                          _p(ranges, C.c_uint32), _p(toff, C.c_int64))
    keys = np.zeros(max(total, 1), np.uint64)
    vals = np.zeros(max(total, 1), np.uint32)
    lib().orc_bin(C.c_int32(V), C.c_int64(n), _p(uv32, C.c_float), _p(radius, C.c_int32), _p(depth32, C.c_float),
                  _p(Ws, C.c_int32), _p(Hs, C.c_int32), C.c_int32(tile[0]), C.c_int32(tile[1]),
                  _p(keys, C.c_uint64), _p(vals, C.c_uint32), C.c_int64(total), _p(ranges, C.c_uint32),
                  _p(toff, C.c_int64))
    return Bins(keys=keys[:total], values=vals[:total], ranges=ranges[:nt], tile_offset=toff)


def decision_inputs(projs: List[Projected]):
    """Float32 decision inputs of the binning from the float64 projection (rounded once)."""
    uv32 = np.stack([p.uv for p in projs]).astype(np.float32)
    rad = np.stack([p.radius for p in projs]).astype(np.int32)
    d32 = np.stack([p.depth for p in projs]).astype(np.float32)
    return uv32, rad, d32


# ----------------------------------------------------------------------------------------
@dataclass
class Render:
    images: List[np.ndarray]    # per view [H, W, 4] (RGB + T bg, alpha = 1 - T)
    final_T: List[np.ndarray]   # per view [H, W]
    last: List[np.ndarray]      # per view [H, W] uint32
    margins: List[np.ndarray]   # per view [H, W, N_MARGINS]
    projs: List[Projected]
    bins: Bins
    comp: Composed
    table: np.ndarray


def render(models, edits, cams, bg=(0.0, 0.0, 0.0), tile=(16, 16), lowpass: float = LOWPASS,
           comp: Optional[Composed] = None, table: Optional[np.ndarray] = None) -> Render:
    comp = compose(models) if comp is None else comp
    table = edit_table(edits) if table is None else table
    bg = np.ascontiguousarray(bg, np.float64)
    projs = [project(comp, table, c, lowpass) for c in cams]
    bins = bin_pairs(*decision_inputs(projs), [(c.W, c.H) for c in cams], tile)
    imgs, Ts, lasts, margins = [], [], [], []
    for v, (c, p) in enumerate(zip(cams, projs)):
        rgba = np.zeros((c.H, c.W, 4))
        T = np.zeros((c.H, c.W))
        last = np.zeros((c.H, c.W), np.uint32)
        mg = np.zeros((c.H, c.W, N_MARGINS))
        lib().orc_render_view(_p(p.uv), _p(p.conic), _p(p.opacity), _p(p.rgb), _p(bins.values, C.c_uint32),
                              _p(bins.ranges, C.c_uint32), C.c_int64(int(bins.tile_offset[v])), C.c_int32(c.W),
                              C.c_int32(c.H), C.c_int32(tile[0]), C.c_int32(tile[1]), _p(bg), _p(rgba), _p(T),
                              _p(last, C.c_uint32), _p(mg))
        imgs.append(rgba); Ts.append(T); lasts.append(last); margins.append(mg)
    return Render(imgs, Ts, lasts, margins, projs, bins, comp, table)


@dataclass
class Grads:
    params: dict              # name -> float64 array, same shape as the composed attribute
    edit: np.ndarray          # same layout as the edit table
    light: np.ndarray         # [V, 3]
    proj: List[dict]          # per view: uv, conic, opacity, rgb gradients


def render_backward(r: Render, cams, dL_drgba: Sequence[np.ndarray], bg=(0.0, 0.0, 0.0), tile=(16, 16),
                    lowpass: float = LOWPASS) -> Grads:
    comp, table = r.comp, r.table
    bg = np.ascontiguousarray(bg, np.float64)
    n = comp.n
    params = _grad_params(comp)
    dedit = np.zeros_like(table)
    dlight = np.zeros((len(cams), 3))
    per_view = []
    for v, (c, p) in enumerate(zip(cams, r.projs)):
        g = dict(uv=np.zeros((n, 2)), conic=np.zeros((n, 3)), opacity=np.zeros(n), rgb=np.zeros((n, 3)))
        d = np.ascontiguousarray(dL_drgba[v], np.float64)
        lib().orc_render_view_backward(_p(p.uv), _p(p.conic), _p(p.opacity), _p(p.rgb),
                                       _p(r.bins.values, C.c_uint32), _p(r.bins.ranges, C.c_uint32),
                                       C.c_int64(int(r.bins.tile_offset[v])), C.c_int32(c.W), C.c_int32(c.H),
                                       C.c_int32(tile[0]), C.c_int32(tile[1]), _p(bg), _p(d), _p(g["uv"]),
                                       _p(g["conic"]), _p(g["opacity"]), _p(g["rgb"]))
        _project_backward(comp, table, c, lowpass, g, params, dedit, dlight[v])
        per_view.append(g)
    return Grads(params, dedit, dlight, per_view)


def _sh_args(comp):
    if comp.sh is None:
        return (None, C.c_int32(-1))
    return (_p(np.ascontiguousarray(comp.sh, np.float64)), C.c_int32(comp.sh_degree))


def _grad_params(comp):
    params = {k: np.zeros_like(getattr(comp, k)) for k in PARAMS}
    if comp.sh is not None:
        params["sh"] = np.zeros_like(comp.sh, np.float64)
    return params


def _project_backward(comp, table, cam, lowpass, g, params, dedit, dlight_v):
    oc = camera(cam)
    d_sh = params.get("sh")
    lib().orc_project_backward(C.c_int64(comp.n), *[_p(a) for a in comp.arrays()], _p(comp.model_id, C.c_int32),
                               *_sh_args(comp), _p(table), C.c_int32(comp.n_models), C.byref(oc),
                               C.c_double(lowpass), C.c_double(GUARD), _p(g["uv"]), _p(g["conic"]), _p(g["opacity"]),
                               _p(g["rgb"]), *[_p(params[k]) for k in PARAMS], _p(d_sh) if d_sh is not None else None,
                               _p(dedit), _p(dlight_v))


# ----------------------------------------------------------------------------------------
# Sampled pixels at full size: each pixel's list is built directly from the definition
# (every Gaussian whose float32 rectangle covers the pixel's tile, ordered by (depth bits,
# index)), so no full-image binning is needed.
# ----------------------------------------------------------------------------------------
def pixel_lists(p: Projected, cam, pix: np.ndarray, tile=(16, 16)):
    uv32 = p.uv.astype(np.float32)
    r = p.radius.astype(np.float32)
    gx = (cam.W + tile[0] - 1) // tile[0]
    gy = (cam.H + tile[1] - 1) // tile[1]
    tw, th = np.float32(tile[0]), np.float32(tile[1])
    x0 = np.clip(np.floor((uv32[:, 0] - r) / tw), 0, gx)
    x1 = np.clip(np.floor((uv32[:, 0] + r) / tw) + np.float32(1), 0, gx)
    y0 = np.clip(np.floor((uv32[:, 1] - r) / th), 0, gy)
    y1 = np.clip(np.floor((uv32[:, 1] + r) / th) + np.float32(1), 0, gy)
    live = p.radius > 0
    bits = p.depth.astype(np.float32).view(np.uint32)
    offs = [0]
    lists = []
    for (i, j) in pix:
        tx, ty = i // tile[0], j // tile[1]
        sel = np.nonzero(live & (x0 <= tx) & (tx < x1) & (y0 <= ty) & (ty < y1))[0]
        order = np.lexsort((sel, bits[sel]))
        lists.append(sel[order].astype(np.uint32))
        offs.append(offs[-1] + len(sel))
    flat = np.concatenate(lists) if lists else np.zeros(0, np.uint32)
    return np.asarray(offs, np.int64), np.ascontiguousarray(flat, np.uint32)


def render_pixels(p: Projected, cam, pix: np.ndarray, bg=(0.0, 0.0, 0.0), tile=(16, 16)):
    """Composite the sampled pixels pix[k] = (i, j) of one view; returns rgba, T, last, margins."""
    pix = np.asarray(pix, np.int64).reshape(-1, 2)
    offs, flat = pixel_lists(p, cam, pix, tile)
    npx = pix.shape[0]
    pxy = np.ascontiguousarray(pix.astype(np.float64) + 0.5)
    rgba = np.zeros((npx, 4)); T = np.zeros(npx); last = np.zeros(npx, np.uint32); mg = np.zeros((npx, N_MARGINS))
    bg = np.ascontiguousarray(bg, np.float64)
    lib().orc_render_pixels(_p(p.uv), _p(p.conic), _p(p.opacity), _p(p.rgb), C.c_int64(npx), _p(pxy),
                            _p(offs, C.c_int64), _p(flat, C.c_uint32), _p(bg), _p(rgba), _p(T),
                            _p(last, C.c_uint32), _p(mg))
    return rgba, T, last, mg


def pixels_backward(comp, table, cams, projs, pix_per_view, dL_per_view, bg=(0.0, 0.0, 0.0), tile=(16, 16),
                    lowpass: float = LOWPASS) -> Grads:
    """Gradients of a loss that touches only the sampled pixels (full-size gradient checks)."""
    n = comp.n
    bg = np.ascontiguousarray(bg, np.float64)
    params = _grad_params(comp)
    dedit = np.zeros_like(table)
    dlight = np.zeros((len(cams), 3))
    per_view = []
    for v, (c, p) in enumerate(zip(cams, projs)):
        g = dict(uv=np.zeros((n, 2)), conic=np.zeros((n, 3)), opacity=np.zeros(n), rgb=np.zeros((n, 3)))
        pix = np.asarray(pix_per_view[v], np.int64).reshape(-1, 2)
        if pix.shape[0]:
            offs, flat = pixel_lists(p, c, pix, tile)
            pxy = np.ascontiguousarray(pix.astype(np.float64) + 0.5)
            d = np.ascontiguousarray(dL_per_view[v], np.float64)
            lib().orc_render_pixels_backward(_p(p.uv), _p(p.conic), _p(p.opacity), _p(p.rgb), C.c_int64(pix.shape[0]),
                                             _p(pxy), _p(offs, C.c_int64), _p(flat, C.c_uint32), _p(bg), _p(d),
                                             _p(g["uv"]), _p(g["conic"]), _p(g["opacity"]), _p(g["rgb"]))
            _project_backward(comp, table, c, lowpass, g, params, dedit, dlight[v])
        per_view.append(g)
    return Grads(params, dedit, dlight, per_view)


# ----------------------------------------------------------------------------------------
# Auxiliary maps (Sec. 4.2 depth / normal maps, Sec. 4.3 offset-colour and coefficient maps,
# the attribute render modes of Sec. 4.7): the RGB blend weights T_i alpha_i applied to
# per-Gaussian values instead of colours.
# ----------------------------------------------------------------------------------------
AUX_CHANNELS = ("depth", "nx", "ny", "nz", "dc_r", "dc_g", "dc_b", "ka", "kd", "ks", "beta")


def aux_attributes(comp: Composed, table: np.ndarray, p: Projected) -> np.ndarray:
    """[N, 11]: camera depth, unit normal (world), offset colour dc, edited k' = lambda k + b."""
    M = comp.n_models
    lam = table[M * EDIT_STRIDE:M * EDIT_STRIDE + 4]
    bias = table[M * EDIT_STRIDE + 4:M * EDIT_STRIDE + 8]
    nrm = comp.normal / np.linalg.norm(comp.normal, axis=1, keepdims=True)
    return np.ascontiguousarray(np.c_[p.depth, nrm, comp.dcolor, comp.kads * lam + bias], np.float64)


def render_aux(r: "Render", cams, tile=(16, 16)) -> List[np.ndarray]:
    """Per view [H, W, 12]: the 11 auxiliary channels (AUX_CHANNELS) and 1 - T."""
    out = []
    for v, (c, p) in enumerate(zip(cams, r.projs)):
        aux = aux_attributes(r.comp, r.table, p)
        o = np.zeros((c.H, c.W, len(AUX_CHANNELS) + 1))
        lib().orc_render_view_aux(_p(p.uv), _p(p.conic), _p(p.opacity), _p(p.rgb), _p(aux),
                                  C.c_int32(len(AUX_CHANNELS)), _p(r.bins.values, C.c_uint32),
                                  _p(r.bins.ranges, C.c_uint32), C.c_int64(int(r.bins.tile_offset[v])),
                                  C.c_int32(c.W), C.c_int32(c.H), C.c_int32(tile[0]), C.c_int32(tile[1]), _p(o))
        out.append(o)
    return out


def render_aux_backward(r: "Render", cams, dL_daux: Sequence[np.ndarray], tile=(16, 16),
                        lowpass: float = LOWPASS) -> Grads:
    """Reverse mode of ``render_aux``: dL_daux[v] is [H, W, 12], the gradient of a loss on the
    11 auxiliary channels and 1 - T. Returns the gradients of the stored attributes and of the
    edit table; ``proj[v]["aux"]`` holds the per-Gaussian [N, 11] channel gradients of view v.

    The auxiliary maps composite the per-Gaussian values x_i with the weights T_i alpha_i and no
    background (Sec. 4.2 first equation), so their reverse mode is the compositing's with x in
    place of the colour and bg = 0. That reverse mode is linear in the upstream gradient: the
    channels are taken three at a time through the float64 compositing reverse mode of
    ``render_backward`` (the 1 - T channel with the first three) and the contributions summed.
    The 2D-quantity gradients then go through the projection's reverse mode with a zero colour
    gradient (Sec. 3 first equation); the channels' own gradients through x_i: the camera depth
    z = (R mu + t)_z, the unit normal n / |n|, the offset colour dc, and k' = lambda k + b."""
    comp, table = r.comp, r.table
    n, M = comp.n, comp.n_models
    params = _grad_params(comp)
    dedit = np.zeros_like(table)
    dlight = np.zeros((len(cams), 3))
    lam = table[M * EDIT_STRIDE:M * EDIT_STRIDE + 4]
    nlen = np.linalg.norm(comp.normal, axis=1, keepdims=True)
    nhat = comp.normal / nlen
    zero_bg = np.zeros(3)
    per_view = []
    for v, (c, p) in enumerate(zip(cams, r.projs)):
        x = aux_attributes(comp, table, p)
        d = np.asarray(dL_daux[v], np.float64)
        g = dict(uv=np.zeros((n, 2)), conic=np.zeros((n, 3)), opacity=np.zeros(n), rgb=np.zeros((n, 3)))
        dx = np.zeros((n, len(AUX_CHANNELS)))
        for k0 in range(0, len(AUX_CHANNELS), 3):
            ks = list(range(k0, min(k0 + 3, len(AUX_CHANNELS))))
            cols = np.zeros((n, 3))
            cols[:, :len(ks)] = x[:, ks]
            dl = np.zeros((c.H, c.W, 4))
            dl[..., :len(ks)] = d[..., ks]
            if k0 == 0:
                dl[..., 3] = d[..., len(AUX_CHANNELS)]
            gk = dict(uv=np.zeros((n, 2)), conic=np.zeros((n, 3)), opacity=np.zeros(n), rgb=np.zeros((n, 3)))
            lib().orc_render_view_backward(_p(p.uv), _p(p.conic), _p(p.opacity), _p(np.ascontiguousarray(cols)),
                                           _p(r.bins.values, C.c_uint32), _p(r.bins.ranges, C.c_uint32),
                                           C.c_int64(int(r.bins.tile_offset[v])), C.c_int32(c.W), C.c_int32(c.H),
                                           C.c_int32(tile[0]), C.c_int32(tile[1]), _p(zero_bg),
                                           _p(np.ascontiguousarray(dl)), _p(gk["uv"]), _p(gk["conic"]),
                                           _p(gk["opacity"]), _p(gk["rgb"]))
            for key in ("uv", "conic", "opacity"):
                g[key] += gk[key]
            dx[:, ks] += gk["rgb"][:, :len(ks)]
        _project_backward(comp, table, c, lowpass, g, params, dedit, dlight[v])
        R = np.asarray(c.R, np.float64).reshape(3, 3)
        params["mean"] += dx[:, 0:1] * R[2][None, :]
        dn = dx[:, 1:4]
        params["normal"] += (dn - nhat * (nhat * dn).sum(1, keepdims=True)) / nlen
        params["dcolor"] += dx[:, 4:7]
        dk = dx[:, 7:11]
        params["kads"] += dk * lam[None, :]
        dedit[M * EDIT_STRIDE:M * EDIT_STRIDE + 4] += (comp.kads * dk).sum(0)
        dedit[M * EDIT_STRIDE + 4:M * EDIT_STRIDE + 8] += dk.sum(0)
        per_view.append(dict(g, aux=dx))
    return Grads(params, dedit, dlight, per_view)

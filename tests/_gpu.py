"""GPU-side harness shared by the `-m gpu` tests (and the smoke check).

Runs the CUDA path through the C ABI (``paper_2504_17954_gb300``) and compares it with the
FP64 oracle under the certification rules for float32-vs-float64 near-ties of
``oracle/certify.py`` (re-exported here): uncertain records (radius, rectangle edge, depth
rounding, near plane) and excused pixels (the oracle's own near-tie record, or a tile touched by
an uncertain record). The number of excused pixels is returned so tests can bound it.
"""
from __future__ import annotations

import contextlib
from typing import List

import numpy as np

import oracle
import scenegen as sg
from oracle.certify import (DEPTH_MARGIN, MARGIN, NEAR_MARGIN, RADIUS_MARGIN, RECT_MARGIN_PX,  # noqa: F401
                            compare_image, depth_uncertain, near_plane_uncertain, near_tie,
                            uncertain_records, uncertain_tile_mask)
from paper_2504_17954_gb300 import Gaussians, Rasterizer, compose_edit

IMG_TOL = 2e-4


def device_models(models) -> List[Gaussians]:
    out = []
    for m in models:
        out.append(Gaussians.from_arrays({k: getattr(m, k) for k in sg.ATTRS}, n_models=1))
    return out


def setup(w: sg.Workload, capacity=None, edits=None, cull=True, tile_h=16):
    ed = w.edits if edits is None else edits
    dm = device_models(w.models)
    comp, table = compose_edit(dm, ed.palette, ed.opacity_scale, ed.visible, ed.lam, ed.bias,
                               light_dir=getattr(ed, "light_dir", None))
    rast = Rasterizer(w.cameras, comp.n, len(w.models), capacity=capacity, lowpass=w.lowpass, bg=w.bg, cull=cull,
                      tile_h=tile_h)
    return rast, comp, table


def last_gaussian(rast: Rasterizer, v: int, pix: np.ndarray) -> np.ndarray:
    """Gaussian index of each sampled pixel's last contributor (-1 if none), from the GPU's
    `last` (a position in the pixel's tile run) and its tile lists; unlike the position it does
    not depend on which non-contributing entries a list holds."""
    c = rast.cams[v]
    th = rast.tile_h
    gx = (c.W + 15) // 16
    t0 = sum(((q.W + 15) // 16) * ((q.H + th - 1) // th) for q in rast.cams[:v])
    last = rast.view_image(v, rast.last).cpu().numpy()[pix[:, 1], pix[:, 0]].astype(np.int64)
    tile = t0 + (pix[:, 1] // th) * gx + pix[:, 0] // 16
    start = rast.ranges.cpu().numpy().view(np.uint32)[tile, 0].astype(np.int64)
    vals = rast.values.cpu().numpy().view(np.uint32).astype(np.int64)
    out = np.full(len(pix), -1, np.int64)
    has = last > 0
    out[has] = vals[start[has] + last[has] - 1]
    return out


def oracle_last_gaussian(offs: np.ndarray, lists: np.ndarray, last: np.ndarray) -> np.ndarray:
    """The same for the oracle's per-pixel lists (oracle.pixel_lists) and its `last`."""
    out = np.full(len(last), -1, np.int64)
    has = last > 0
    out[has] = lists[offs[:-1][has] + last[has].astype(np.int64) - 1]
    return out


def gpu_keys(rast: Rasterizer):
    """The GPU's sorted pairs as 64-bit keys (tile << 32 | depth bits), values and ranges.

    The library returns sorted tile ids; the depth bits of each pair are read back from the
    projected record it refers to, so the keys compare bit for bit with the oracle's."""
    n = rast.n_pairs
    t = rast.tiles[:n].cpu().numpy().view(np.uint32).astype(np.uint64)
    v = rast.values[:n].cpu().numpy().view(np.uint32)
    r = rast.ranges.cpu().numpy().view(np.uint32)
    th = rast.tile_h
    toff = np.cumsum([0] + [((c.W + 15) // 16) * ((c.H + th - 1) // th) for c in rast.cams])
    view = np.searchsorted(toff, t.astype(np.int64), side="right") - 1
    depth = rast.rgbd[:, 3].contiguous().cpu().numpy().view(np.uint32)
    bits = depth[view * rast.n + v.astype(np.int64)].astype(np.uint64)
    k = (t << np.uint64(32)) | bits
    return k, v, r


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / den) if den > 0 else float(np.linalg.norm(a))


GRAD_TOL = 1e-3


def grad_errors(got, want):
    """(relative L2 error ||g - g*|| / ||g*||, largest element error max |g - g*| / max |g*|)."""
    want = np.asarray(want, np.float64)
    got = np.asarray(got, np.float64).reshape(want.shape)
    den = np.linalg.norm(want)
    l2 = float(np.linalg.norm(got - want) / den) if den > 0 else float(np.linalg.norm(got))
    mx = float(np.abs(want).max(initial=0.0))
    d = float(np.abs(got - want).max(initial=0.0))
    el = d / mx if mx > 0 else d
    return l2, el


def assert_grad(got, want, what, tol=GRAD_TOL):
    """The gradient bar: relative L2 error per tensor and every element's error, relative to the
    tensor's largest entry, both within tol."""
    l2, el = grad_errors(got, want)
    assert l2 <= tol and el <= tol, f"{what}: relative L2 {l2:.2e}, element-wise {el:.2e} of max |g*| (bar {tol:.0e})"
    return l2, el


@contextlib.contextmanager
def sequential_walk():
    """Both blends with one CTA per tile (ivrgs option render_split = 2): the split walk regroups
    the float32 transmittance products by chunk, so bit-identity checks between two renders (or
    against the auxiliary maps' sequential walk) hold only for the sequential walk."""
    from paper_2504_17954_gb300 import _native as N
    old = N.ivrgs_get_option("render_split")
    N.ivrgs_set_option("render_split", 2)
    try:
        yield
    finally:
        N.ivrgs_set_option("render_split", old)

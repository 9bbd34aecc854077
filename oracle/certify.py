"""Certification of float32-vs-float64 near-ties (test infrastructure: used by the tests and the
benchmark's oracle leg; the product never imports it).

The GPU path decides in float32, the oracle in float64. A discrete decision may legitimately go
the other way only where the oracle's float64 quantity lies within rounding of its threshold:

* a Gaussian-view record is *uncertain* when its float64 radius 3 sqrt(lambda_max) lies within
  1e-5 (relative) of an integer, or an edge (u +- r) of its tile rectangle lies within 1e-3 px
  of a tile boundary (its tile membership may differ), when its float64 camera depth lies
  within 2^-40 (relative to |t_z| + sum |R_zk mu_k|) of a float32 rounding midpoint (its place
  in the depth order may differ), or within 1e-6 of the near plane;
* a pixel is *excused* from the image tolerance only if the oracle's own decision record for it
  shows a near-tie (|ln(255 alpha)|, |ln(T'/1e-4)| or the relative |P| below 1e-3) or it lies
  in a tile touched (one tile of slack) by an uncertain record.
"""
from __future__ import annotations

import math

import numpy as np

from . import Projected

MARGIN = 1e-3
RADIUS_MARGIN = 1e-5
RECT_MARGIN_PX = 1e-3
DEPTH_MARGIN = 2.0 ** -40
NEAR_MARGIN = 1e-6
ZNEAR = 0.2


def depth_uncertain(p: Projected) -> np.ndarray:
    """Live records whose float32 sort key may legitimately differ from the oracle's."""
    return (p.radius > 0) & (p.depth_margin < DEPTH_MARGIN)


def near_plane_uncertain(p: Projected, znear: float = ZNEAR) -> np.ndarray:
    """Records that either side may cull at the near plane (the oracle's float64 z is within
    NEAR_MARGIN of it); their footprint is unknown where the oracle culled them."""
    return np.abs(p.depth - znear) < NEAR_MARGIN


def uncertain_records(p: Projected, tile: int = 16, tile_h: int = None) -> np.ndarray:
    """Records whose float32 decisions may legitimately differ from the oracle's, for tiles of
    tile x tile_h pixels (tile_h defaults to tile)."""
    th = tile if tile_h is None else tile_h
    live = p.radius > 0
    unc = live & (p.radius_margin < RADIUS_MARGIN)
    unc |= depth_uncertain(p) | near_plane_uncertain(p)
    r = p.radius.astype(np.float64)
    for e, t in ((p.uv[:, 0] - r, tile), (p.uv[:, 0] + r, tile), (p.uv[:, 1] - r, th), (p.uv[:, 1] + r, th)):
        q = e / t
        d = np.abs(q - np.round(q)) * t
        unc |= live & (d < RECT_MARGIN_PX)
    return unc


def uncertain_tile_mask(p: Projected, unc: np.ndarray, W: int, H: int, tile: int = 16,
                        tile_h: int = None) -> np.ndarray:
    th = tile if tile_h is None else tile_h
    gx, gy = (W + tile - 1) // tile, (H + th - 1) // th
    mask = np.zeros((gy, gx), bool)
    if (unc & near_plane_uncertain(p)).any():  # a record at the near plane may cover any pixel
        mask[:] = True
    for g in np.nonzero(unc)[0]:
        u, v = p.uv[g]
        r = p.radius[g] + 1
        x0 = max(int(math.floor((u - r) / tile)) - 1, 0)
        x1 = min(int(math.floor((u + r) / tile)) + 2, gx)
        y0 = max(int(math.floor((v - r) / th)) - 1, 0)
        y1 = min(int(math.floor((v + r) / th)) + 2, gy)
        if x0 < x1 and y0 < y1:
            mask[y0:y1, x0:x1] = True
    return np.kron(mask, np.ones((th, tile), bool))[:H, :W]


def uncertain_pixels(p: Projected, unc: np.ndarray, pix: np.ndarray, margin: float = 1e-2) -> np.ndarray:
    """The pixels pix[k] = (i, j) that an uncertain record reaches: its float64 alpha o' exp(P)
    at the pixel centre is at least (1/255) e^-margin. A record changes a pixel's compositing only
    through its alpha there (below the cut-off both sides skip it, wherever it is listed), so a
    float32 decision about an uncertain record (its tile membership, radius or depth order) can
    only show at these pixels; a record uncertain at the near plane may cover any pixel. Finer
    than uncertain_tile_mask, which excuses every pixel of every tile the record touches."""
    pix = np.asarray(pix, np.int64).reshape(-1, 2)
    out = np.zeros(len(pix), bool)
    if len(pix) == 0:
        return out
    if (unc & near_plane_uncertain(p)).any():
        out[:] = True
        return out
    cx = pix[:, 0].astype(np.float64) + 0.5
    cy = pix[:, 1].astype(np.float64) + 0.5
    cut = math.log(1.0 / 255.0) - margin
    for g in np.nonzero(unc & (p.opacity > 0))[0]:
        a, b, c = p.conic[g]
        dx = p.uv[g, 0] - cx
        dy = p.uv[g, 1] - cy
        P = -0.5 * (a * dx * dx + 2.0 * b * dx * dy + c * dy * dy)
        out |= P + math.log(p.opacity[g]) >= cut
    return out


def near_tie(margins: np.ndarray) -> np.ndarray:
    return (margins[..., 0] < MARGIN) | (margins[..., 1] < MARGIN) | (margins[..., 2] < MARGIN)


def compare_image(gpu: np.ndarray, ref: np.ndarray, margins: np.ndarray, extra_excuse=None, tol=2e-4):
    """Returns (max error over non-excused pixels, number excused, number of pixels over tol)."""
    err = np.abs(gpu.astype(np.float64) - ref).max(-1)
    over = err > tol
    ok_excuse = near_tie(margins)
    if extra_excuse is not None:
        ok_excuse |= extra_excuse
    bad = over & ~ok_excuse
    excused = over & ok_excuse
    strict = np.where(excused, 0.0, err)
    return float(strict.max()) if strict.size else 0.0, int(excused.sum()), int(bad.sum())

"""Brute-force per-pixel compositing for tiny scenes (test infrastructure only).

For every pixel it scans ALL Gaussians, keeps those whose float32 tile rectangle covers the
pixel's tile, orders them by (float32 depth, index) and composites them front to back with the
second equation of Sec. 3 and the 0.99 / (1/255) / 1e-4 thresholds.  It uses no tile lists, no
binning and no sort of keys, so agreement with the tiled oracle pins the binning and ordering.
The transmittance in front of each Gaussian is formed as an explicit product over the ones
already composited (not carried as a running variable).
"""
from __future__ import annotations

import math

import numpy as np


def render_view(uv, conic, opacity, rgb, depth, radius, W, H, bg=(0.0, 0.0, 0.0), tile=16):
    uv32 = uv.astype(np.float32)
    r = radius.astype(np.float32)
    gx, gy = (W + tile - 1) // tile, (H + tile - 1) // tile
    t = np.float32(tile)
    x0 = np.clip(np.floor((uv32[:, 0] - r) / t), 0, gx)
    x1 = np.clip(np.floor((uv32[:, 0] + r) / t) + np.float32(1), 0, gx)
    y0 = np.clip(np.floor((uv32[:, 1] - r) / t), 0, gy)
    y1 = np.clip(np.floor((uv32[:, 1] + r) / t) + np.float32(1), 0, gy)
    live = radius > 0
    bits = depth.astype(np.float32).view(np.uint32)
    out = np.zeros((H, W, 4))
    for j in range(H):
        for i in range(W):
            tx, ty = i // tile, j // tile
            sel = np.nonzero(live & (x0 <= tx) & (tx < x1) & (y0 <= ty) & (ty < y1))[0]
            sel = sel[np.lexsort((sel, bits[sel]))]
            alphas, cols = [], []
            for g in sel:
                dx = uv[g, 0] - (i + 0.5)
                dy = uv[g, 1] - (j + 0.5)
                a, b, c = conic[g]
                P = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
                if P > 0:
                    continue
                al = min(0.99, opacity[g] * math.exp(P))
                if al < 1.0 / 255.0:
                    continue
                T_next = math.prod(1.0 - x for x in alphas) * (1.0 - al)
                if T_next < 1e-4:
                    break
                alphas.append(al)
                cols.append(rgb[g])
            col = np.zeros(3)
            for k, (al, cc) in enumerate(zip(alphas, cols)):
                col += math.prod(1.0 - x for x in alphas[:k]) * al * np.asarray(cc)
            T = math.prod(1.0 - x for x in alphas)
            out[j, i, :3] = col + T * np.asarray(bg)
            out[j, i, 3] = 1.0 - T
    return out

"""FP64 oracle of inverse volume exploration (Sec. 4.6) -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may use this module;
the product never does, and it shares no code with the CUDA path.

* ``image_loss``: the loss the paper fits a composed model to a reference image with, read as
  the 3DGS loss its "combination of L1 and SSIM" refers to: (1 - lambda) L1 + lambda (1 - SSIM)
  over R, G, B of every view; L1 = mean |x - y|; SSIM (Wang et al. 2004) per pixel and channel
  with an 11 x 11 Gaussian window (sigma 1.5, normalised), C1 = 0.01^2, C2 = 0.03^2 and zero
  padding at each view's border, averaged over all pixels and channels. The windowed sums are
  a library 2D correlation with the full window; the gradient is the chain rule of those
  definitions written out.
* ``adam_step``: Adam (Kingma and Ba 2015) with bias-corrected moments,
  step = lr m^ / (sqrt(v^) + eps), on the learnable edit-table values (Sec. 4.6: per-model c_p
  and opacity scale, global lambda and b) and on the global light's polar / azimuthal angles,
  dir = (sin t cos p, sin t sin p, cos t).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np
from scipy import ndimage

C1 = 0.01 ** 2
C2 = 0.03 ** 2
EDIT_STRIDE = 8
LEARN_COLOR, LEARN_OPACITY, LEARN_LIGHT_MAGNITUDE, LEARN_LIGHT_DIRECTION = 1, 2, 4, 8


def ssim_window() -> np.ndarray:
    """11 x 11 Gaussian window, sigma 1.5, weights summing to 1."""
    k = np.arange(-5, 6, dtype=np.float64)
    g = np.exp(-(k[:, None] ** 2 + k[None, :] ** 2) / (2 * 1.5 ** 2))
    return g / g.sum()


def _wsum(img: np.ndarray) -> np.ndarray:
    """Windowed sum with zero padding outside the image (library 2D correlation)."""
    return ndimage.correlate(img, ssim_window(), mode="constant", cval=0.0)


def ssim_map(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Per-pixel SSIM of two single-channel images."""
    mx, my = _wsum(x), _wsum(y)
    sxx = _wsum(x * x) - mx * mx
    syy = _wsum(y * y) - my * my
    sxy = _wsum(x * y) - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def _ssim_grad(x: np.ndarray, y: np.ndarray, g: float) -> np.ndarray:
    """d(g * sum_q S(q))/dx for single-channel images (g = dL/dS, the same for every q)."""
    mx, my = _wsum(x), _wsum(y)
    sxx = _wsum(x * x) - mx * mx
    syy = _wsum(y * y) - my * my
    sxy = _wsum(x * y) - mx * my
    A1, A2 = 2 * mx * my + C1, 2 * sxy + C2
    B1, B2 = mx * mx + my * my + C1, sxx + syy + C2
    S = A1 * A2 / (B1 * B2)
    dS_dmx = 2 * my * A2 / (B1 * B2) - S * 2 * mx / B1   # at fixed sigmas
    dS_dsxx = -S / B2
    dS_dsxy = 2 * A1 / (B1 * B2)
    # total derivatives w.r.t. the windowed sums E[x] = mx, E[x^2], E[xy]
    d_Ex = dS_dmx - 2 * mx * dS_dsxx - my * dS_dsxy
    d_Exx = dS_dsxx
    d_Exy = dS_dsxy
    # E[f](q) = sum_p w(q - p) f(p): the adjoint is the correlation with the flipped window,
    # which is the same window (symmetric)
    return g * (_wsum(d_Ex) + 2 * x * _wsum(d_Exx) + y * _wsum(d_Exy))


def image_loss(xs: Sequence[np.ndarray], ys: Sequence[np.ndarray], lam: float = 0.2
               ) -> Tuple[float, float, float, List[np.ndarray]]:
    """xs, ys: per view [H, W, >=3] images. Returns (loss, L1, SSIM, [dloss/dx per view, [H, W, 3]])."""
    n = sum(3 * x.shape[0] * x.shape[1] for x in xs)
    l1 = sum(np.abs(x[..., :3] - y[..., :3]).sum() for x, y in zip(xs, ys)) / n
    ssim = sum(ssim_map(x[..., c].astype(np.float64), y[..., c].astype(np.float64)).sum()
               for x, y in zip(xs, ys) for c in range(3)) / n
    grads = []
    for x, y in zip(xs, ys):
        gr = np.zeros(x.shape[:2] + (3,))
        for c in range(3):
            xc, yc = x[..., c].astype(np.float64), y[..., c].astype(np.float64)
            gr[..., c] = (1 - lam) * np.sign(xc - yc) / n + _ssim_grad(xc, yc, -lam / n)
        grads.append(gr)
    return (1 - lam) * l1 + lam * (1 - ssim), l1, ssim, grads


# ---------------------------------------------------------------------------------------
def light_dir(polar: float, azimuth: float) -> np.ndarray:
    return np.array([np.sin(polar) * np.cos(azimuth), np.sin(polar) * np.sin(azimuth), np.cos(polar)])


def light_angles(d: np.ndarray) -> Tuple[float, float]:
    d = np.asarray(d, np.float64)
    return float(np.arccos(np.clip(d[2] / np.linalg.norm(d), -1.0, 1.0))), float(np.arctan2(d[1], d[0]))


class AdamState:
    """First / second moments per learnable value, the light angles and the step count."""

    def __init__(self, table: np.ndarray, n_models: int):
        P = 4 * n_models + 10
        self.m = np.zeros(P)
        self.v = np.zeros(P)
        L = table[n_models * EDIT_STRIDE + 8:n_models * EDIT_STRIDE + 11]
        self.angles = np.array(light_angles(L)) if np.linalg.norm(L) > 0 else np.zeros(2)
        self.t = 0


def adam_step(table: np.ndarray, egrad: np.ndarray, n_models: int, st: AdamState, learn: int, lr: float,
              b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8) -> np.ndarray:
    """One Adam step; returns the new table (the state is updated in place). egrad has the
    edit-gradient layout (table-shaped; the global light's slots hold dloss/d dir)."""
    M = n_models
    tab = np.array(table, np.float64, copy=True)
    st.t += 1
    idx, grads, learnable = [], [], []
    for j in range(4 * M):
        m, k = divmod(j, 4)
        idx.append(m * EDIT_STRIDE + k)
        grads.append(egrad[m * EDIT_STRIDE + k])
        learnable.append(bool(learn & (LEARN_COLOR if k < 3 else LEARN_OPACITY)))
    for k in range(8):
        idx.append(M * EDIT_STRIDE + k)
        grads.append(egrad[M * EDIT_STRIDE + k])
        learnable.append(bool(learn & LEARN_LIGHT_MAGNITUDE))
    th, ph = st.angles
    gd = egrad[M * EDIT_STRIDE + 8:M * EDIT_STRIDE + 11]
    on = tab[M * EDIT_STRIDE + 11] != 0.0
    dth = np.dot(gd, [np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)])
    dph = np.dot(gd, [-np.sin(th) * np.sin(ph), np.sin(th) * np.cos(ph), 0.0])
    idx += [None, None]
    grads += [dth, dph]
    learnable += [bool(learn & LEARN_LIGHT_DIRECTION) and on] * 2
    for j, (i, g, ok) in enumerate(zip(idx, grads, learnable)):
        if not ok:
            continue
        st.m[j] = b1 * st.m[j] + (1 - b1) * g
        st.v[j] = b2 * st.v[j] + (1 - b2) * g * g
        mh = st.m[j] / (1 - b1 ** st.t)
        vh = st.v[j] / (1 - b2 ** st.t)
        step = lr * mh / (np.sqrt(vh) + eps)
        if i is None:
            st.angles[j - 4 * M - 8] -= step
        else:
            tab[i] -= step
    if (learn & LEARN_LIGHT_DIRECTION) and on:
        tab[M * EDIT_STRIDE + 8:M * EDIT_STRIDE + 11] = light_dir(*st.angles)
    return tab

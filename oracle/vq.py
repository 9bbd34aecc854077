"""FP64 oracle of the vector-quantised storage (Sec. 4.4) -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may use this module;
it shares no code with the CUDA path. Per basic model, every attribute except the mean and the
normal gets one scalar codebook shared by its components, from k-means (Lloyd's algorithm) on
that model's values of the attribute: k centroids spaced evenly over [min, max]
(c_j = lo + (hi - lo)(j + 0.5)/k), then `iters` rounds of (assign every value to its nearest
centroid, a value exactly on a midpoint to the lower one; move every centroid to the mean of
its values, an empty one stays). Each component then stores the index of its nearest centroid.
"""
from __future__ import annotations

from typing import Dict, Tuple

import numpy as np

# codebooks per model, in storage order; kads component j uses codebook 4 + j
ATTRS = ("log_scale", "quat", "opacity_logit", "dcolor", "k_a", "k_d", "k_s", "beta")


def nearest(cent: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Index of the nearest of the sorted centroids; on a midpoint the lower one."""
    mids = 0.5 * (cent[:-1] + cent[1:])
    return np.searchsorted(mids, v, side="left")


def kmeans_1d(values: np.ndarray, k: int, iters: int) -> np.ndarray:
    v = np.asarray(values, np.float64).ravel()
    lo, hi = (float(v.min()), float(v.max())) if v.size else (0.0, 0.0)
    cent = lo + (hi - lo) * (np.arange(k) + 0.5) / k
    for _ in range(iters):
        j = nearest(cent, v)
        s = np.bincount(j, weights=v, minlength=k)
        n = np.bincount(j, minlength=k)
        cent = np.where(n > 0, s / np.maximum(n, 1), cent)
        cent = np.maximum.accumulate(cent)
    return cent


def _attr_values(arrs: Dict[str, np.ndarray], sel: np.ndarray, a: int) -> np.ndarray:
    name = ATTRS[a]
    if a >= 4:
        return arrs["kads"][sel, a - 4]
    return arrs[name][sel]


def build(arrs: Dict[str, np.ndarray], model_id: np.ndarray, n_models: int, k: int, iters: int
          ) -> Tuple[np.ndarray, Dict[str, np.ndarray]]:
    """codebook [n_models, 8, k] (float64) and uint8 indices per attribute array."""
    n = len(model_id)
    cb = np.zeros((n_models, len(ATTRS), k))
    idx = {"log_scale": np.zeros((n, 3), np.uint8), "quat": np.zeros((n, 4), np.uint8),
           "opacity_logit": np.zeros(n, np.uint8), "dcolor": np.zeros((n, 3), np.uint8),
           "kads": np.zeros((n, 4), np.uint8)}
    for m in range(n_models):
        sel = np.nonzero(model_id == m)[0]
        for a in range(len(ATTRS)):
            vals = _attr_values(arrs, sel, a).astype(np.float64)
            cb[m, a] = kmeans_1d(vals, k, iters) if sel.size else np.zeros(k)
            j = nearest(cb[m, a], vals).astype(np.uint8)
            if a >= 4:
                idx["kads"][sel, a - 4] = j
            else:
                idx[ATTRS[a]][sel] = j.reshape(idx[ATTRS[a]][sel].shape)
    return cb, idx


def decode(cb: np.ndarray, idx: Dict[str, np.ndarray], model_id: np.ndarray) -> Dict[str, np.ndarray]:
    m = model_id.astype(np.int64)
    out = {"log_scale": cb[m[:, None], 0, idx["log_scale"]], "quat": cb[m[:, None], 1, idx["quat"]],
           "opacity_logit": cb[m, 2, idx["opacity_logit"]], "dcolor": cb[m[:, None], 3, idx["dcolor"]],
           "kads": np.stack([cb[m, 4 + j, idx["kads"][:, j]] for j in range(4)], 1)}
    return out

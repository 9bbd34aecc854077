"""Writes the regression fixture ``oracle_two_models_40x24.json`` beside this script.

The fixture freezes one small composed scene (inputs, stored exactly) together with what the
FP64 oracle computes for it: the float32-decided tile lists (Sec. 3, tile-based rasterization),
sampled pixels and per-channel sums of both views' images (Sec. 3, front-to-back compositing
with the shading of Sec. 3's Blinn-Phong model and the edits of Sec. 4.5-4.6), and the full
reverse mode for a closed-form dL/dRGBA. Every stored value is written by this script through
``oracle/`` alone; the inputs come from ``scenegen``.

The fixture is a regression record of the oracle, not a pin of it (the pins are the
``tests/test_oracle_*.py`` checks against closed forms, brute force and finite differences):
``tests/test_golden.py`` recomputes it and fails on any change of the oracle's arithmetic,
which then has to be justified by the passage of the paper it follows before this script is
re-run.

    python tests/golden/make_golden.py
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(_HERE)))

import oracle  # noqa: E402
import scenegen as sg  # noqa: E402

NAME = "oracle_two_models_40x24.json"
MODEL_KEYS = sg.ATTRS + ("palette",)
CAMERA_KEYS = ("W", "H", "fx", "fy", "cx", "cy", "R", "t", "campos", "znear", "headlight", "light_dir")
EDIT_KEYS = ("palette", "opacity_scale", "visible", "lam", "bias")
# dL/dRGBA of view v at pixel (x, y), channel c; a closed form so that the fixture stays small
DL_FORMULA = "sin(0.7 x + 1.3 y + 2.1 c + 0.5 v)"
N_SAMPLES = 48


def dl_drgba(W: int, H: int, v: int) -> np.ndarray:
    y, x, c = np.meshgrid(np.arange(H), np.arange(W), np.arange(4), indexing="ij")
    return np.sin(0.7 * x + 1.3 * y + 2.1 * c + 0.5 * v)


def sample_pixels(W: int, H: int, v: int) -> np.ndarray:
    """N_SAMPLES distinct pixel indices of one view, spread over the image (a fixed stride)."""
    step = max(1, (W * H) // N_SAMPLES)
    return (np.arange(N_SAMPLES) * step + 7 * v) % (W * H)


def scene() -> sg.Workload:
    """Two basic models (9 + 7 Gaussians, large enough to straddle tiles), random edits, a
    headlight view and an orbital-light view of 40 x 24 pixels (3 x 2 tiles, ragged), both close
    enough for the scene to reach every tile."""
    base = sg.tiny_scene(16, 40, 24, 71, log_scale_mu=-2.0, n_models=2)
    r = np.random.default_rng(72)
    head = sg.look_at(1.5 * sg.random_direction(r), 40, 24)
    orbital = sg.look_at(1.5 * sg.random_direction(r), 40, 24, headlight=False,
                         light_dir=sg.random_direction(r).astype(np.float32))
    ed = sg.random_edits(base.models, seed=73)
    ed.lam = np.array([1.1, 0.9, 1.2, 0.8], np.float32)
    ed.bias = np.array([0.02, -0.01, 0.03, 0.5], np.float32)
    return sg.Workload("golden", base.models, [head, orbital], ed, bg=np.array([0.2, 0.1, 0.3], np.float32))


def _plain(x):
    a = np.asarray(x)
    return a.tolist() if a.ndim else a.item()


def inputs_json(w: sg.Workload) -> dict:
    return {
        "models": [{k: _plain(getattr(m, k)) for k in MODEL_KEYS} for m in w.models],
        "cameras": [{k: _plain(getattr(c, k)) for k in CAMERA_KEYS} for c in w.cameras],
        "edits": {k: _plain(getattr(w.edits, k)) for k in EDIT_KEYS},
        "bg": _plain(w.bg),
    }


def workload_from(inp: dict) -> sg.Workload:
    """The stored inputs as a Workload (float32 arrays, exactly the values written)."""
    f32 = lambda a: np.asarray(a, np.float32)
    models = [sg.Model(**{k: f32(d[k]) for k in MODEL_KEYS}) for d in inp["models"]]
    cams = []
    for d in inp["cameras"]:
        cams.append(sg.Camera(W=int(d["W"]), H=int(d["H"]), fx=d["fx"], fy=d["fy"], cx=d["cx"], cy=d["cy"],
                              R=f32(d["R"]), t=f32(d["t"]), campos=f32(d["campos"]), znear=d["znear"],
                              headlight=int(d["headlight"]), light_dir=f32(d["light_dir"])))
    e = inp["edits"]
    ed = sg.Edits(palette=f32(e["palette"]), opacity_scale=f32(e["opacity_scale"]),
                  visible=np.asarray(e["visible"], np.int32), lam=f32(e["lam"]), bias=f32(e["bias"]))
    return sg.Workload("golden", models, cams, ed, bg=f32(inp["bg"]))


# a float32 evaluation may decide differently from the FP64 oracle only near a tie: a radius
# 3 sqrt(lambda_max) within 1e-5 (relative) of an integer, a rectangle edge within 1e-3 px of a
# tile boundary, a camera depth within 2^-40 (relative) of a float32 rounding midpoint or within
# 1e-6 of the near plane (the record refuses such scenes), or a pixel whose alpha cut-off,
# termination or P > 0 decision is within 1e-3 (relative) of its threshold (flagged per pixel)
RADIUS_TIE, EDGE_TIE_PX, DEPTH_TIE, NEAR_TIE, PIXEL_TIE = 1e-5, 1e-3, 2.0 ** -40, 1e-6, 1e-3


def check_no_record_ties(p) -> None:
    live = p.radius > 0
    r = p.radius.astype(np.float64)
    near = live & (p.radius_margin < RADIUS_TIE)
    near |= live & (p.depth_margin < DEPTH_TIE)
    near |= np.abs(p.depth - sg.ZNEAR) < NEAR_TIE
    for e in (p.uv[:, 0] - r, p.uv[:, 0] + r, p.uv[:, 1] - r, p.uv[:, 1] + r):
        q = e / 16.0
        near |= live & (np.abs(q - np.round(q)) * 16.0 < EDGE_TIE_PX)
    if near.any():
        raise ValueError(f"records {np.flatnonzero(near).tolist()} sit at a float32 decision tie")


def outputs(w: sg.Workload) -> dict:
    """What the oracle computes for the scene: the fixture's expected values."""
    ref = oracle.render(w.models, w.edits, w.cameras, bg=w.bg)
    for p in ref.projs:
        check_no_record_ties(p)
    dls = [dl_drgba(c.W, c.H, v) for v, c in enumerate(w.cameras)]
    g = oracle.render_backward(ref, w.cameras, dls, bg=w.bg)
    views = []
    for v, c in enumerate(w.cameras):
        img = ref.images[v]
        pix = sample_pixels(c.W, c.H, v)
        views.append({
            "uv32": _plain(ref.projs[v].uv.astype(np.float32)),
            "radius": _plain(ref.projs[v].radius),
            "depth32": _plain(ref.projs[v].depth.astype(np.float32)),
            "pixels": _plain(pix),
            "rgba": _plain(img.reshape(-1, 4)[pix]),
            "last": _plain(ref.last[v].reshape(-1)[pix]),
            "near_tie": _plain((ref.margins[v].reshape(-1, oracle.N_MARGINS)[pix, :3] < PIXEL_TIE).any(1)),
            "rgba_sum": _plain(img.reshape(-1, 4).sum(0)),
        })
    return {
        "tile_offset": _plain(ref.bins.tile_offset),
        "ranges": _plain(ref.bins.ranges),
        "values": _plain(ref.bins.values),
        "views": views,
        "grad": {k: _plain(g.params[k]) for k in oracle.PARAMS},
        "grad_edit": _plain(g.edit),
        "grad_light": _plain(g.light),
    }


def main():
    w = scene()
    inp = inputs_json(w)
    doc = {
        "what": "one composed scene and the FP64 oracle's results for it (regression record)",
        "cite": "Sec. 3 (EWA projection, Blinn-Phong shading, tiled front-to-back compositing), "
                "Sec. 4.3 (editable attributes), Sec. 4.5-4.6 (composition and edits)",
        "written_by": "tests/golden/make_golden.py (oracle/ only)",
        "dL_drgba": DL_FORMULA,
        "inputs": inp,
        # computed from the stored inputs, so the record holds exactly what they give
        "outputs": outputs(workload_from(inp)),
    }
    with open(os.path.join(_HERE, NAME), "w") as f:
        json.dump(doc, f, separators=(",", ":"))
        f.write("\n")


if __name__ == "__main__":
    main()

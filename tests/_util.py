"""Small constructors shared by the tests (hand-built scenes and cameras)."""
from __future__ import annotations

import math

import numpy as np

import scenegen as sg


def axis_camera(W=32, H=32, z=3.0, f=None, headlight=True, light_dir=None) -> sg.Camera:
    """Camera with R = I (camera axes = world axes) placed at (0, 0, -z), looking along +z."""
    f = sg.focal_for(H) if f is None else f
    ld = np.zeros(3, np.float32) if light_dir is None else np.asarray(light_dir, np.float32)
    return sg.Camera(W=W, H=H, fx=float(np.float32(f)), fy=float(np.float32(f)), cx=W / 2.0, cy=H / 2.0,
                     R=np.eye(3, dtype=np.float32).reshape(9), t=np.array([0, 0, z], np.float32),
                     campos=np.array([0, 0, -z], np.float32), headlight=1 if headlight else 0, light_dir=ld)


def single_model(mean, log_scale=(-4.0, -4.0, -4.0), quat=(1, 0, 0, 0), logit=0.0, albedo=(0.5, 0.5, 0.5),
                 normal=(0, 0, -1), kads=sg.KADS_DEFAULT, palette=None) -> sg.Model:
    a = np.asarray(albedo, np.float64)
    cp = a if palette is None else np.asarray(palette, np.float64)
    f32 = lambda x, shape: np.asarray(x, np.float32).reshape(shape)
    return sg.Model(mean=f32(mean, (1, 3)), log_scale=f32(log_scale, (1, 3)), quat=f32(quat, (1, 4)),
                    opacity_logit=f32([logit], (1,)), dcolor=f32(a - cp, (1, 3)), normal=f32(normal, (1, 3)),
                    kads=f32(kads, (1, 4)), palette=f32(cp, (3,)))


def cat_models(ms):
    keys = sg.ATTRS
    out = sg.Model(**{k: np.concatenate([getattr(m, k) for m in ms]) for k in keys},
                   palette=ms[0].palette.copy())
    return out


def logit(p: float) -> float:
    return math.log(p / (1.0 - p))

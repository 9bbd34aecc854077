"""Seeded synthetic inputs shared by the oracle-side tests, the GPU tests and the benchmark.

This module only draws inputs. It holds no step of the rendering method (no projection,
shading, binning, sorting or compositing): every number here is either a random draw or a
camera/scene definition that both the oracle and the CUDA path consume as given.

Scene recipe (a stand-in for Gaussians fitted to value bands of a volume, Sec. 4 of the paper
composes one basic model per disjoint transfer-function band):

* Scalar field f(x) = sum_k exp(-|x - c_k|^2 / (2 w_k^2)), c_k ~ U[-0.7, 0.7]^3,
  w_k ~ U[0.15, 0.35], normalised by its maximum over a 128^3 grid of [-1, 1]^3.
* A basic model takes points x ~ U[-1, 1]^3 with f(x) inside its band (a 0.5 +- 0.02 shell
  for the single-model workloads; equal-width bands over [0.05, 0.95] for composed ones).
  Sampling is exact rejection from the grid voxels whose corner values come within 0.02 of
  the band, so the accepted points are uniform over the band region.
* Per Gaussian: log-scale ~ N(-4.5, 0.5)^3, quaternion uniform on S^3 (normalised N(0,1)^4,
  stored (w, x, y, z)), opacity logit ~ N(0, 1.5), albedo ~ U[0, 1]^3, normal uniform on S^2,
  (k_a, k_d, k_s, beta) = (0.2, 0.7, 0.3, 32).
* Editable colour (Sec. 4.3): the palette colour c_p of a model is the mean albedo of its
  Gaussians, and the per-Gaussian offset is dc = albedo - c_p.
* Cameras: pinhole, world->camera rotation R (rows: right, down, forward), t = -R campos,
  f_x = f_y = (H/2)/tan(22.5 deg), principal point (W/2, H/2), looking at the origin from
  radius 3 with world up +z (+y when forward is parallel to +z).

All arrays are float32 (the values the GPU path stores); the oracle reads the same values
exactly as float64.  Seeds: 0 scenes, 1 cameras, 2 edits, 3 perturbations, 4 FD picks.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

KADS_DEFAULT = (0.2, 0.7, 0.3, 32.0)
FOV_Y_DEG = 45.0
ZNEAR = 0.2
ATTRS = ("mean", "log_scale", "quat", "opacity_logit", "dcolor", "normal", "kads")


def _rng(*key: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(list(key))))


# ----------------------------------------------------------------------------------------
# scalar field and band sampling
# ----------------------------------------------------------------------------------------
@dataclass
class BlobField:
    centres: np.ndarray  # [K, 3] float64
    widths: np.ndarray   # [K]
    norm: float = 1.0
    grid: Optional[np.ndarray] = None  # [G, G, G] normalised samples (corner values)

    def __call__(self, x: np.ndarray) -> np.ndarray:
        x = np.asarray(x, dtype=np.float64)
        out = np.zeros(x.shape[0], dtype=np.float64)
        step = 1 << 18
        inv = 1.0 / (2.0 * self.widths ** 2)
        cc = (self.centres ** 2).sum(1)
        for s in range(0, x.shape[0], step):
            xs = x[s:s + step]
            d2 = (xs ** 2).sum(1)[:, None] - 2.0 * xs @ self.centres.T + cc[None, :]
            out[s:s + step] = np.exp(-np.maximum(d2, 0.0) * inv[None, :]).sum(1)
        return out / self.norm


def blob_field(n_blobs: int, seed: int = 0, grid: int = 128) -> BlobField:
    r = _rng(seed, 1000 + n_blobs)
    f = BlobField(centres=r.uniform(-0.7, 0.7, (n_blobs, 3)), widths=r.uniform(0.15, 0.35, n_blobs))
    ax = np.linspace(-1.0, 1.0, grid)
    pts = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
    vals = f(pts)
    f.norm = float(vals.max())
    f.grid = (vals / f.norm).reshape(grid, grid, grid)
    return f


def sample_band(f: BlobField, lo: float, hi: float, count: int, rng: np.random.Generator,
                margin: float = 0.02) -> np.ndarray:
    """Uniform points of [-1,1]^3 with lo <= f(x) <= hi, by rejection inside candidate voxels."""
    g = f.grid
    n = g.shape[0]
    h = 2.0 / (n - 1)
    corners = [g[a:n - 1 + a, b:n - 1 + b, c:n - 1 + c] for a in (0, 1) for b in (0, 1) for c in (0, 1)]
    vmin = np.minimum.reduce(corners)
    vmax = np.maximum.reduce(corners)
    cand = np.argwhere((vmax >= lo - margin) & (vmin <= hi + margin))
    if cand.shape[0] == 0:
        raise ValueError(f"band [{lo}, {hi}] is empty")
    out = np.empty((0, 3))
    while out.shape[0] < count:
        need = count - out.shape[0]
        batch = max(4096, int(need * 2.5))
        vox = cand[rng.integers(0, cand.shape[0], batch)]
        x = -1.0 + (vox + rng.random((batch, 3))) * h
        v = f(x)
        out = np.concatenate([out, x[(v >= lo) & (v <= hi)]], 0)
    return out[:count]


# ----------------------------------------------------------------------------------------
# editable Gaussians (Sec. 4.3 attribute set)
# ----------------------------------------------------------------------------------------
@dataclass
class Model:
    mean: np.ndarray
    log_scale: np.ndarray
    quat: np.ndarray
    opacity_logit: np.ndarray
    dcolor: np.ndarray
    normal: np.ndarray
    kads: np.ndarray
    palette: np.ndarray  # c_p, [3]

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    def copy(self) -> "Model":
        return Model(**{k: np.array(getattr(self, k), copy=True) for k in ATTRS + ("palette",)})


def make_model(centres: np.ndarray, rng: np.random.Generator) -> Model:
    n = centres.shape[0]
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    nrm = rng.standard_normal((n, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    albedo = rng.random((n, 3))
    palette = albedo.mean(0)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Model(
        mean=f32(centres),
        log_scale=f32(rng.normal(-4.5, 0.5, (n, 3))),
        quat=f32(q),
        opacity_logit=f32(rng.normal(0.0, 1.5, n)),
        dcolor=f32(albedo - palette),
        normal=f32(nrm),
        kads=f32(np.tile(np.array(KADS_DEFAULT), (n, 1))),
        palette=f32(palette),
    )


# ----------------------------------------------------------------------------------------
# cameras
# ----------------------------------------------------------------------------------------
@dataclass
class Camera:
    W: int
    H: int
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray        # [9] float32 world->camera, row-major
    t: np.ndarray        # [3] float32
    campos: np.ndarray   # [3] float32
    znear: float = ZNEAR
    headlight: int = 1
    light_dir: np.ndarray = field(default_factory=lambda: np.zeros(3, np.float32))

    @property
    def npix(self) -> int:
        return self.W * self.H


def focal_for(H: int, fov_y_deg: float = FOV_Y_DEG) -> float:
    return (H / 2.0) / math.tan(math.radians(fov_y_deg) / 2.0)


def look_at(campos, W: int, H: int, target=(0.0, 0.0, 0.0), headlight: bool = True,
            light_dir=None) -> Camera:
    c = np.asarray(campos, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - c
    fwd /= np.linalg.norm(fwd)
    up = np.array([0.0, 0.0, 1.0])
    right = np.cross(fwd, up)
    if np.linalg.norm(right) < 1e-6:
        right = np.cross(fwd, np.array([0.0, 1.0, 0.0]))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd], 0).astype(np.float32)
    t = (-(R.astype(np.float64) @ c)).astype(np.float32)
    campos32 = (-(R.astype(np.float64).T @ t.astype(np.float64))).astype(np.float32)
    f = focal_for(H)
    ld = np.zeros(3, np.float32) if light_dir is None else np.asarray(light_dir, np.float32)
    return Camera(W=W, H=H, fx=float(np.float32(f)), fy=float(np.float32(f)),
                  cx=float(np.float32(W / 2.0)), cy=float(np.float32(H / 2.0)),
                  R=R.reshape(9), t=t, campos=campos32, headlight=1 if headlight else 0, light_dir=ld)


def fibonacci_sphere(n: int, radius: float = 3.0) -> np.ndarray:
    i = np.arange(n) + 0.5
    z = 1.0 - 2.0 * i / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    return radius * np.stack([r * np.cos(phi), r * np.sin(phi), z], 1)


def random_direction(rng: np.random.Generator) -> np.ndarray:
    d = rng.standard_normal(3)
    return d / np.linalg.norm(d)


def orbital_light(polar_deg: float, azimuth_rad: float) -> np.ndarray:
    """Unit vector towards a directional light at elevation `polar_deg` and a given azimuth."""
    th = math.radians(polar_deg)
    return np.array([math.cos(th) * math.cos(azimuth_rad), math.cos(th) * math.sin(azimuth_rad),
                     math.sin(th)], dtype=np.float32)


# ----------------------------------------------------------------------------------------
# edits (Sec. 4.5 / 4.6): per-model palette, opacity scale, visibility; global lambda, b
# ----------------------------------------------------------------------------------------
@dataclass
class Edits:
    palette: np.ndarray        # [M, 3]
    opacity_scale: np.ndarray  # [M]
    visible: np.ndarray        # [M] int32
    lam: np.ndarray = field(default_factory=lambda: np.ones(4, np.float32))
    bias: np.ndarray = field(default_factory=lambda: np.zeros(4, np.float32))
    light_dir: Optional[np.ndarray] = None  # one orbital light direction for every view, or None

    def copy(self) -> "Edits":
        return Edits(*(np.array(a, copy=True) for a in (self.palette, self.opacity_scale,
                                                        self.visible, self.lam, self.bias)),
                     light_dir=None if self.light_dir is None else np.array(self.light_dir, copy=True))


def identity_edits(models: List[Model]) -> Edits:
    return Edits(palette=np.stack([m.palette for m in models]).astype(np.float32),
                 opacity_scale=np.ones(len(models), np.float32),
                 visible=np.ones(len(models), np.int32))


def random_edits(models: List[Model], seed: int = 2, hide: Optional[int] = None) -> Edits:
    r = _rng(seed, 77)
    M = len(models)
    vis = np.ones(M, np.int32)
    if hide is not None:
        vis[hide] = 0
    return Edits(palette=r.random((M, 3)).astype(np.float32),
                 opacity_scale=r.uniform(0.3, 1.5, M).astype(np.float32), visible=vis)


# ----------------------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    models: List[Model]
    cameras: List[Camera]
    edits: Edits
    bg: np.ndarray = field(default_factory=lambda: np.zeros(3, np.float32))
    tile: int = 16
    lowpass: float = 0.3

    @property
    def n_gaussians(self) -> int:
        return sum(m.n for m in self.models)

    @property
    def n_pixels(self) -> int:
        return sum(c.npix for c in self.cameras)


def _cache_path(key: str) -> Optional[str]:
    root = os.environ.get("IVRGS_SCENE_CACHE")
    if not root:
        return None
    os.makedirs(root, exist_ok=True)
    return os.path.join(root, key + ".npz")


def make_models(n_blobs: int, bands, counts, seed: int = 0) -> List[Model]:
    key = f"models_b{n_blobs}_s{seed}_" + "_".join(f"{lo:.4f}-{hi:.4f}x{c}" for (lo, hi), c in zip(bands, counts))
    path = _cache_path(key)
    if path and os.path.exists(path):
        z = np.load(path)
        out = []
        for m in range(len(counts)):
            out.append(Model(**{k: z[f"{m}_{k}"] for k in ATTRS + ("palette",)}))
        return out
    f = blob_field(n_blobs, seed)
    models = []
    for m, ((lo, hi), c) in enumerate(zip(bands, counts)):
        r = _rng(seed, m)
        models.append(make_model(sample_band(f, lo, hi, c, r), r))
    if path:
        np.savez(path, **{f"{m}_{k}": getattr(mod, k) for m, mod in enumerate(models)
                          for k in ATTRS + ("palette",)})
    return models


def equal_bands(n: int, lo: float = 0.05, hi: float = 0.95):
    e = np.linspace(lo, hi, n + 1)
    return [(float(e[i]), float(e[i + 1])) for i in range(n)]


def config1(seed: int = 0) -> Workload:
    """10k Gaussians on the 0.5 shell of an 8-blob field; one 128x128 view; FP32 forward."""
    models = make_models(8, [(0.48, 0.52)], [10_000], seed)
    cam = look_at(3.0 * random_direction(_rng(1, 1)), 128, 128)
    return Workload("cfg1: 10k Gaussians, 1 view 128x128", models, [cam], identity_edits(models))


def config2(seed: int = 0) -> Workload:
    """500k Gaussians on the 0.5 shell of a 32-blob field; one 800x800 view; fwd+bwd."""
    models = make_models(32, [(0.48, 0.52)], [500_000], seed)
    cam = look_at(3.0 * random_direction(_rng(1, 2)), 800, 800)
    return Workload("cfg2: 500k Gaussians, 1 view 800x800", models, [cam], identity_edits(models))


def perturbed(models: List[Model], seed: int = 3) -> List[Model]:
    """Target scene for the L1 loss: positions + N(0, 0.01), albedo jitter U[-0.1, 0.1]."""
    out = []
    for i, m in enumerate(models):
        r = _rng(seed, i)
        c = m.copy()
        c.mean = (m.mean + r.normal(0.0, 0.01, m.mean.shape)).astype(np.float32)
        c.dcolor = (m.dcolor + r.uniform(-0.1, 0.1, m.dcolor.shape)).astype(np.float32)
        out.append(c)
    return out


def config3(seed: int = 0) -> Workload:
    """6 composed models (1.5M), 16 views at 1024^2 with an orbital light sweep; forward."""
    counts = [80_000, 150_000, 220_000, 300_000, 350_000, 400_000]
    models = make_models(64, equal_bands(6), counts, seed)
    pos = fibonacci_sphere(16)
    cams = []
    for i, p in enumerate(pos):
        az = math.atan2(p[1], p[0])
        cams.append(look_at(p, 1024, 1024, headlight=False,
                            light_dir=orbital_light(-90.0 + 180.0 * i / 15.0, az)))
    return Workload("cfg3: 1.5M Gaussians / 6 models, 16 views 1024x1024", models, cams,
                    random_edits(models, hide=2))


CFG4_SIZES = [(512, 512), (800, 800), (1024, 768), (1280, 1280)]


def config4(seed: int = 0, n_views: int = 8) -> Workload:
    """4 composed models (1M), 8 views of uneven sizes; forward + backward."""
    counts = [100_000, 200_000, 300_000, 400_000]
    models = make_models(64, equal_bands(4), counts, seed)
    pos = fibonacci_sphere(n_views)
    cams = [look_at(p, *CFG4_SIZES[i % 4]) for i, p in enumerate(pos)]
    return Workload("cfg4: 1M Gaussians / 4 models, 8 views 512^2..1280^2", models, cams,
                    identity_edits(models))


def config4_two_views(seed: int = 0) -> Workload:
    """The 1M-Gaussian scene of config4 seen by its first two views (512^2, 800^2): a profiling
    case whose buffers stay around 1 GB while its pair arrays exceed the L2 cache."""
    w = config4(seed)
    w.cameras = w.cameras[:2]
    w.name = "cfg4-2v: 1M Gaussians / 4 models, 2 views 512^2 + 800^2"
    return w


def config5(seed: int = 0, n_views: int = 64) -> Workload:
    """8 composed models (3M, counts 1:2:..:8), 64 views with sides ~ U{512..2048}."""
    w = np.arange(1, 9)
    counts = [int(3_000_000 * k / w.sum()) for k in w]
    counts[-1] += 3_000_000 - sum(counts)
    models = make_models(64, equal_bands(8), counts, seed)
    r = _rng(1, 5)
    sides = r.integers(512, 2049, n_views)
    pos = fibonacci_sphere(n_views)
    cams = [look_at(p, int(s), int(s)) for p, s in zip(pos, sides)]
    return Workload("cfg5: 3M Gaussians / 8 models, 64 views 512^2..2048^2", models, cams,
                    random_edits(models))


def fd_subscene(seed: int = 0, n: int = 200, size: int = 64) -> Workload:
    """Small scene for finite-difference checks: 200 Gaussians, one 64x64 view.

    Scales are raised (log-scale ~ N(-3.2, 0.3)) so that the Gaussians cover the small image.
    """
    f = blob_field(8, seed)
    r = _rng(seed, 500)
    x = sample_band(f, 0.48, 0.52, n, r)
    m = make_model(x, r)
    m.log_scale = r.normal(-3.2, 0.3, (n, 3)).astype(np.float32)
    cam = look_at(3.0 * random_direction(_rng(1, 4)), size, size)
    return Workload("fd: 200 Gaussians, 64x64", [m], [cam], identity_edits([m]))


def tiny_scene(n: int, W: int, H: int, seed: int, log_scale_mu: float = -3.0,
               headlight: bool = True, n_models: int = 1) -> Workload:
    """Tiny random scene for brute-force and invariant checks."""
    r = _rng(seed, 900)
    models = []
    per = [n // n_models + (1 if i < n % n_models else 0) for i in range(n_models)]
    for k in per:
        x = r.uniform(-0.6, 0.6, (k, 3))
        m = make_model(x, r)
        m.log_scale = r.normal(log_scale_mu, 0.3, (k, 3)).astype(np.float32)
        models.append(m)
    cr = _rng(seed, 901)
    light = None if headlight else random_direction(cr).astype(np.float32)
    cam = look_at(3.0 * random_direction(cr), W, H, headlight=headlight, light_dir=light)
    return Workload(f"tiny n={n} {W}x{H}", models, [cam], identity_edits(models))


# ----------------------------------------------------------------------------------------
# synthetic projected records for the binning/sorting checks
# ----------------------------------------------------------------------------------------
def synthetic_projected(sizes, n: int, seed: int, tie_frac: float = 0.3, max_radius: int = 40):
    """Random (u, v, radius, depth) per view for exercising tile binning and the key sort.

    Depths are drawn from a small set of values for a fraction of the entries so that many
    keys tie on depth; about 10% of radii are 0 (culled) and some means lie off-screen.
    """
    r = _rng(seed, 300)
    V = len(sizes)
    xy = np.empty((V, n, 2), np.float32)
    rad = np.empty((V, n), np.int32)
    depth = np.empty((V, n), np.float32)
    for v, (W, H) in enumerate(sizes):
        xy[v, :, 0] = r.uniform(-50, W + 50, n)
        xy[v, :, 1] = r.uniform(-50, H + 50, n)
        rr = r.integers(0, max_radius + 1, n)
        rr[r.random(n) < 0.1] = 0
        rad[v] = rr
        d = r.uniform(0.25, 6.0, n)
        tie = r.random(n) < tie_frac
        d[tie] = r.choice(np.array([1.0, 2.5, 3.0, 3.25]), tie.sum())
        depth[v] = d
    return xy, rad, depth


# ----------------------------------------------------------------------------------------
# 16-bit storage encoding (an input format, not a step of the rendering method)
# ----------------------------------------------------------------------------------------
ANCHOR_CHUNK = 256


def _spread10(x):
    x = x.astype(np.uint32) & np.uint32(0x3FF)
    x = (x | (x << np.uint32(16))) & np.uint32(0x030000FF)
    x = (x | (x << np.uint32(8))) & np.uint32(0x0300F00F)
    x = (x | (x << np.uint32(4))) & np.uint32(0x030C30C3)
    x = (x | (x << np.uint32(2))) & np.uint32(0x09249249)
    return x


def to_bf16_bits(a) -> np.ndarray:
    """float32 -> bfloat16 bit patterns, round to nearest even (finite inputs)."""
    b = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = (b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    return r.astype(np.uint16)


def bf16_bits_to_f32(bits) -> np.ndarray:
    return (np.asarray(bits, np.uint16).astype(np.uint32) << np.uint32(16)).view(np.float32)


def morton_order(mean, model_id, lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0)) -> np.ndarray:
    """The memory layout of a composed set: indices sorted (stably) by (model id, 30-bit Morton
    code of the float32 mean quantised to 1024 steps per axis inside the box [lo, hi])."""
    mean = np.ascontiguousarray(mean, np.float32)
    lo32, hi32 = np.asarray(lo, np.float32), np.asarray(hi, np.float32)
    inv = (np.float32(1.0) / (hi32 - lo32)).astype(np.float32)
    q = np.clip((mean - lo32) * inv * np.float32(1024.0), np.float32(0.0), np.float32(1023.0)).astype(np.uint32)
    code = (_spread10(q[:, 0]) << np.uint32(2)) | (_spread10(q[:, 1]) << np.uint32(1)) | _spread10(q[:, 2])
    key = (np.asarray(model_id).astype(np.uint64) << np.uint64(30)) | code.astype(np.uint64)
    return np.argsort(key, kind="stable")


def pack_mixed_arrays(mean, log_scale, quat, opacity_logit, dcolor, normal, kads, model_id,
                      lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0)):
    """The 16-bit storage of concatenated float32 attributes: reorder by (model id, Morton code
    of the mean in the box [lo, hi], index), one float32 anchor per chunk of 256 at the centre
    of the chunk's bounding box, FP16 mean offsets, BF16 log-scale / colour offset / normal,
    FP16 quaternion / opacity logit / k. Returns (dict of arrays, order)."""
    f = lambda a: np.ascontiguousarray(a, np.float32)
    mean, log_scale, quat, dcolor, normal, kads = map(f, (mean, log_scale, quat, dcolor, normal, kads))
    opacity_logit = f(opacity_logit)
    order = morton_order(mean, model_id, lo, hi)
    n = len(order)
    m = mean[order]
    n_chunks = (n + ANCHOR_CHUNK - 1) // ANCHOR_CHUNK
    anchor = np.zeros((max(n_chunks, 1), 3), np.float32)
    off = np.zeros((n, 3), np.float16)
    for c in range(n_chunks):
        sl = slice(c * ANCHOR_CHUNK, min(n, (c + 1) * ANCHOR_CHUNK))
        a = (np.float32(0.5) * (m[sl].min(0) + m[sl].max(0))).astype(np.float32)
        anchor[c] = a
        off[sl] = (m[sl] - a).astype(np.float32).astype(np.float16)
    out = dict(mean=off, anchor=anchor, log_scale=to_bf16_bits(log_scale[order]), quat=quat[order].astype(np.float16),
               opacity_logit=opacity_logit[order].astype(np.float16), dcolor=to_bf16_bits(dcolor[order]),
               normal=to_bf16_bits(normal[order]), kads=kads[order].astype(np.float16),
               model_id=np.asarray(model_id)[order].astype(np.int16))
    return out, order


def decode_mixed_arrays(p):
    """Float32 values of the 16-bit storage: mean = float32(anchor + offset), the rest widened."""
    n = p["mean"].shape[0]
    anchor = np.repeat(p["anchor"], ANCHOR_CHUNK, 0)[:n]
    return dict(mean=(anchor + p["mean"].astype(np.float32)).astype(np.float32),
                log_scale=bf16_bits_to_f32(p["log_scale"]), quat=p["quat"].astype(np.float32),
                opacity_logit=p["opacity_logit"].astype(np.float32), dcolor=bf16_bits_to_f32(p["dcolor"]),
                normal=bf16_bits_to_f32(p["normal"]), kads=p["kads"].astype(np.float32))

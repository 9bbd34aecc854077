"""Autotuner for the library's launch shapes and the batch shape of many-view rendering.

``tune`` searches the options ``ivrgs_set_option`` accepts (pixels per thread of the forward and
backward blend, the split walk of long runs over CTA clusters and its chunk length, radix
ranking and offsets) on the caller's own workload with CUDA events: coordinate descent from the
current setting, one option at a time over all its values, repeated until a sweep changes
nothing (at most ``sweeps`` times). ``tune_waves`` picks the tile height and the view-wave shape
of a ``WaveRasterizer`` (pixels and views per binning call) by timing the caller's whole step
for each distinct shape. Choices are cached in a JSON file keyed by GPU name and a workload
signature. Every option and shape gives the same results (up to float32 rounding in the split
walk), so tuning changes speed only.
"""
from __future__ import annotations

import json
import os
from typing import Callable, Dict, Optional, Sequence

import torch

from . import _native as N

SPACE = {
    "render_pixels_per_thread": (0, 1, 2, 4, 8),
    "render_bwd_pixels_per_thread": (0, 1, 2, 4, 8),
    "render_split": (0, 1, 2, 3, 4),
    "render_split_min": (128, 256, 384, 768, 1024),
    "sort_match": (0, 1),
    "sort_scan": (0, 1),
    "sort_early": (0, 1),
}


# pixel budgets of a view wave: up to 2^16 tiles of 16 x 16 per binning call at 16M pixels (tile
# ids sort in two 8-bit passes as 16-bit keys), more above it (three passes); fewer pixels per
# wave mean more calls and launches
WAVE_BUDGETS = (8 << 20, 16 << 20, 32 << 20)
WAVE_VIEWS = (32,)
# tile heights (tiles are 16 pixels wide): 8-pixel-high tiles shorten each tile's list and the
# walk of a heavy tile, for more pairs to bin and sort
TILE_HEIGHTS = (16, 8)


def _cache_path() -> str:
    return os.environ.get("IVRGS_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache",
                                                                "ivrgs_autotune.json"))


def current() -> Dict[str, int]:
    return {k: N.ivrgs_get_option(k) for k in SPACE}


def apply(choice: Dict[str, int]):
    for k, v in choice.items():
        N.ivrgs_set_option(k, int(v))


def time_ms(step: Callable[[], None], reps: int = 5) -> float:
    """Median device time of one call of ``step`` (CUDA events on the current stream)."""
    step()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        step()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ts.sort()
    return ts[len(ts) // 2]


def tune(step: Callable[[], None], signature: str, reps: int = 5, use_cache: bool = True,
         space: Optional[Dict[str, tuple]] = None, sweeps: int = 2) -> Dict[str, int]:
    """Pick the fastest option combination for ``step`` and apply it.

    ``signature`` names the workload (sizes, views); the result is cached per GPU name."""
    space = SPACE if space is None else space
    key = f"{torch.cuda.get_device_name()}|{signature}"
    path = _cache_path()
    cache = _load_cache(path) if use_cache else {}
    if use_cache and key in cache:
        choice = cache[key]["choice"]
        apply(choice)
        return choice
    names = list(space)
    start = current()
    best = {k: start[k] if start.get(k) in space[k] else space[k][0] for k in names}
    apply(best)
    seen = {}

    def measure(choice):
        sig = tuple(choice[k] for k in names)
        if sig not in seen:
            apply(choice)
            seen[sig] = time_ms(step, reps)
        return seen[sig]
    best_ms = default_ms = measure(best)
    for _ in range(sweeps):
        changed = False
        for k in names:
            for val in space[k]:
                trial = dict(best, **{k: val})
                t = measure(trial)
                if t < best_ms:
                    best, best_ms, changed = trial, t, True
        if not changed:
            break
    apply(best)
    if use_cache:
        cache[key] = {"choice": best, "ms": best_ms, "default_ms": default_ms, "evaluated": len(seen)}
        _store_cache(path, cache)
    return best


def _load_cache(path):
    if os.path.exists(path):
        try:
            with open(path) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}
    return {}


def _store_cache(path, cache):
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass


def tune_waves(measure: Callable[[int, int, int], float], cams: Sequence, n_gaussians: int, signature: str,
               budgets: Sequence[int] = WAVE_BUDGETS, max_views: Sequence[int] = WAVE_VIEWS,
               tile_heights: Sequence[int] = TILE_HEIGHTS, use_cache: bool = True,
               device_name: Optional[str] = None) -> Dict:
    """Pick the tile shape and the view-wave shape of a many-view render for the caller's own step.

    ``measure(max_views, pixel_budget, tile_h)`` builds the waves with that shape (tiles 16
    pixels wide and tile_h high), runs the caller's step (for instance a captured forward+backward
    over all waves) and returns its time in ms; it may raise (a wave over the per-call pair limit,
    out of memory), and that shape is then skipped. Shapes that give the same tile height and wave
    plan (``rasterizer.plan_waves``) are measured once. Returns {"max_views", "pixel_budget",
    "tile_h", "waves" (views per wave), "ms", "candidates" (every measured shape with its time or
    the error)}; cached per GPU name and ``signature``."""
    from .rasterizer import plan_waves
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name()
    key = f"{device_name}|waves|{signature}"
    path = _cache_path()
    cache = _load_cache(path) if use_cache else {}
    if use_cache and key in cache:
        return cache[key]
    plans = {}
    for th in tile_heights:
        for mv in max_views:
            for pb in budgets:
                plan = tuple(len(w) for w in plan_waves(cams, n_gaussians, mv, pb, th))
                plans.setdefault((th, plan), (mv, pb))  # the first shape that gives a plan stands for it
    best = None
    cands = []
    for (th, plan), (mv, pb) in plans.items():
        c = {"max_views": mv, "pixel_budget": pb, "tile_h": th, "waves": list(plan)}
        try:
            ms = float(measure(mv, pb, th))
        except (RuntimeError, MemoryError) as e:
            cands.append(dict(c, error=str(e)[:200]))
            continue
        cands.append(dict(c, ms=ms))
        if best is None or ms < best["ms"]:
            best = dict(c, ms=ms)
    if best is None:
        raise RuntimeError(f"tune_waves: no shape could be measured: {cands}")
    best["candidates"] = cands
    if use_cache:
        cache[key] = best
        _store_cache(path, cache)
    return best

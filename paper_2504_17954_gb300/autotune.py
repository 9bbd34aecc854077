"""Autotuner for the library's launch shapes.

Searches the options ``ivrgs_set_option`` accepts (pixels per thread of the forward and backward
blend, the split walk of long runs over CTA clusters and its chunk length, radix ranking and
offsets) on the caller's own workload with CUDA events: coordinate descent from the current
setting, one option at a time over all its values, repeated until a sweep changes nothing (at
most ``sweeps`` times). The choice is cached in a JSON file keyed by GPU name and a workload
signature. Every option gives the same results (up to float32 rounding in the split walk), so
tuning changes speed only.
"""
from __future__ import annotations

import json
import os
from typing import Callable, Dict, Optional

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
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
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
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return best

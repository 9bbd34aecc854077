"""Autotuner for the library's launch shapes.

Times every combination of the options ``ivrgs_set_option`` accepts (pixels per thread of the
forward and backward blend, radix ranking) on the caller's own workload with CUDA events, keeps
the fastest, and caches the choice in a JSON file keyed by GPU name and a workload signature.
Every option gives the same results, so tuning changes speed only.
"""
from __future__ import annotations

import itertools
import json
import os
from typing import Callable, Dict, Optional

import torch

from . import _native as N

SPACE = {
    "render_pixels_per_thread": (0, 1, 2, 4, 8),
    "render_bwd_pixels_per_thread": (0, 1, 2, 4, 8),
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
         space: Optional[Dict[str, tuple]] = None) -> Dict[str, int]:
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
    before = current()
    results = []
    names = list(space)
    for combo in itertools.product(*(space[k] for k in names)):
        choice = dict(zip(names, combo))
        apply(choice)
        results.append((time_ms(step, reps), choice))
    results.sort(key=lambda r: r[0])
    best = results[0][1]
    apply(best)
    if use_cache:
        cache[key] = {"choice": best, "ms": results[0][0], "default_ms": next(t for t, c in results if c == before)
                      if any(c == before for _, c in results) else None}
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return best

"""CPU tests of the shape autotuner's host logic (paper_2504_17954_gb300.autotune.tune_waves)
with a fake timer: every distinct (tile height, wave plan) is measured once, the fastest shape
wins, a shape whose measurement fails is skipped and reported, and the choice is cached per
signature."""
import json

import pytest

from paper_2504_17954_gb300 import autotune
from paper_2504_17954_gb300.rasterizer import plan_waves


class _Cam:
    def __init__(self, W, H):
        self.W, self.H = W, H


def _cams():
    sides = [512, 2048, 1024, 1536, 2048, 512, 768, 2048, 1024, 1280, 2048, 640]
    return [_Cam(s, s) for s in sides]


def test_each_distinct_plan_is_measured_once_and_the_fastest_wins():
    cams = _cams()
    seen = []

    def measure(mv, pb, th):
        seen.append((mv, pb, th))
        return {8 << 20: 30.0, 16 << 20: 20.0, 32 << 20: 25.0}[pb] + mv * 1e-3 + (3.0 if th == 8 else 0.0)

    best = autotune.tune_waves(measure, cams, 1000, "t", budgets=(8 << 20, 16 << 20, 32 << 20),
                               max_views=(4, 32), tile_heights=(16, 8), use_cache=False, device_name="fake")
    plans = {(th, tuple(len(w) for w in plan_waves(cams, 1000, mv, pb, th))) for mv, pb, th in seen}
    assert len(plans) == len(seen)  # no shape measured twice
    all_plans = {(th, tuple(len(w) for w in plan_waves(cams, 1000, mv, pb, th)))
                 for th in (16, 8) for mv in (4, 32) for pb in (8 << 20, 16 << 20, 32 << 20)}
    assert plans == all_plans
    assert best["tile_h"] == 16
    assert best["ms"] == min(c["ms"] for c in best["candidates"])
    assert best["waves"] == [len(w) for w in plan_waves(cams, 1000, best["max_views"], best["pixel_budget"],
                                                         best["tile_h"])]
    assert sum(best["waves"]) == len(cams)


def test_a_failing_shape_is_skipped_and_reported():
    cams = _cams()

    def measure(mv, pb, th):
        if pb == 16 << 20 and th == 16:
            raise RuntimeError("pair buffer over the per-call limit")
        return (10.0 if pb == 8 << 20 else 12.0) - (1.0 if th == 8 else 0.0)

    best = autotune.tune_waves(measure, cams, 1000, "t", use_cache=False, device_name="fake")
    assert best["pixel_budget"] == 8 << 20 and best["tile_h"] == 8
    errs = [c for c in best["candidates"] if "error" in c]
    assert len(errs) == 1 and errs[0]["pixel_budget"] == 16 << 20 and errs[0]["tile_h"] == 16
    with pytest.raises(RuntimeError):
        autotune.tune_waves(lambda mv, pb, th: (_ for _ in ()).throw(RuntimeError("no")), cams, 1000, "t",
                            use_cache=False, device_name="fake")


def test_choice_is_cached_per_signature(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("IVRGS_AUTOTUNE_CACHE", str(path))
    cams = _cams()
    calls = []

    def measure(mv, pb, th):
        calls.append(pb)
        return float(pb >> 20)

    a = autotune.tune_waves(measure, cams, 1000, "sig", device_name="fake")
    n = len(calls)
    b = autotune.tune_waves(measure, cams, 1000, "sig", device_name="fake")
    assert len(calls) == n and a == b  # from the cache
    autotune.tune_waves(measure, cams, 1000, "other", device_name="fake")
    assert len(calls) == 2 * n
    assert set(json.loads(path.read_text())) == {"fake|waves|sig", "fake|waves|other"}

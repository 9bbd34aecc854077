"""The view-wave plan of WaveRasterizer (host logic, no GPU): many views are rendered in
consecutive waves so that no binning call exceeds the library's limits (IVRGS_MAX_PAIRS
records per call, i.e. n_gaussians * views < 2^30), the caller's pixel budget or 2^16 tiles
(the tile ids' 16-bit sort keys)."""
from types import SimpleNamespace

import numpy as np
import pytest

from paper_2504_17954_gb300 import _native as N
from paper_2504_17954_gb300.rasterizer import n_tiles, plan_waves


def _cams(sizes):
    return [SimpleNamespace(W=int(w), H=int(h)) for w, h in sizes]


def _check(cams, n, max_views, budget, tile_h=16, max_tiles=1 << 16):
    waves = plan_waves(cams, n, max_views, budget, tile_h, max_tiles)
    cap = max(1, min(max_views, (N.IVRGS_MAX_PAIRS - 1) // max(n, 1)))
    assert [v for wv in waves for v in wv] == list(range(len(cams)))  # every view once, in order
    pix = lambda wv: sum(cams[v].W * cams[v].H for v in wv)
    tiles = lambda wv: n_tiles([cams[v] for v in wv], 16, tile_h)
    for i, wv in enumerate(waves):
        assert 1 <= len(wv) <= cap
        assert n * len(wv) < N.IVRGS_MAX_PAIRS or len(wv) == 1
        assert pix(wv) <= budget or len(wv) == 1
        assert tiles(wv) <= max_tiles or len(wv) == 1
        if i + 1 < len(waves):  # greedy: the next view did not fit into this wave
            nxt = waves[i + 1][0]
            assert (len(wv) == cap or pix(wv) + cams[nxt].W * cams[nxt].H > budget
                    or tiles(wv) + tiles([nxt]) > max_tiles)
    return waves


@pytest.mark.parametrize("seed", range(6))
def test_random_plans_respect_every_limit(seed):
    rng = np.random.default_rng(seed)
    V = int(rng.integers(1, 200))
    cams = _cams(rng.integers(16, 2049, (V, 2)))
    n = int(rng.choice([1000, 1_000_000, 3_000_000, 1 << 27, 1 << 29]))
    _check(cams, n, int(rng.integers(1, 80)), int(rng.integers(1 << 18, 1 << 26)), int(rng.choice([16, 8])),
           int(rng.choice([1 << 12, 1 << 16, 1 << 20])))


def test_tile_limit():
    # 2048^2 views hold 16,384 tiles of 16 x 16 (32,768 of 16 x 8): four (two) to a wave of 2^16
    cams = _cams([(2048, 2048)] * 9)
    assert [len(w) for w in _check(cams, 1000, 32, 1 << 30)] == [4, 4, 1]
    assert [len(w) for w in _check(cams, 1000, 32, 1 << 30, tile_h=8)] == [2, 2, 2, 2, 1]
    # a view of more tiles than the limit forms a wave of its own
    assert [len(w) for w in _check(_cams([(64, 64), (4096, 4096), (64, 64)]), 1000, 32, 1 << 30)] == [1, 1, 1]


def test_record_limit_sets_the_wave_size():
    cams = _cams([(64, 64)] * 10)
    # 2^28 Gaussians: 3 views give 3 * 2^28 < 2^30 records, 4 would not
    assert [len(w) for w in _check(cams, 1 << 28, 32, 1 << 30)] == [3, 3, 3, 1]
    # 2^30 - 1 Gaussians or more: one view per wave
    assert [len(w) for w in _check(cams, (1 << 30) - 1, 32, 1 << 30)] == [1] * 10


def test_pixel_budget_and_oversized_views():
    cams = _cams([(1024, 1024), (2048, 2048), (512, 512), (512, 512), (4096, 4096), (16, 16)])
    waves = _check(cams, 1000, 32, 4 << 20)
    # 1 Mpix, then the 4 Mpix view alone (it fills the budget), the two 0.25 Mpix views, the
    # 16 Mpix view alone (larger than the budget), and the last one
    assert waves == [[0], [1], [2, 3], [4], [5]]


def test_max_views_and_empty():
    assert plan_waves([], 1000) == []
    assert [len(w) for w in _check(_cams([(32, 32)] * 70), 1000, 32, 1 << 30)] == [32, 32, 6]

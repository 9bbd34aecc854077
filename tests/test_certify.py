"""CPU tests of the per-pixel near-tie excuse used at full size (oracle/certify.py): an uncertain
record excuses exactly the pixels where its float64 alpha reaches the 1/255 cut-off (with the
stated margin), never a pixel it cannot reach, and always within the coarser tile mask."""
import math

import numpy as np

from oracle import Projected
from oracle.certify import ZNEAR, uncertain_pixels, uncertain_tile_mask


def _records(n):
    return Projected(uv=np.zeros((n, 2)), cov=np.zeros((n, 3)), conic=np.zeros((n, 3)), opacity=np.zeros(n),
                     rgb=np.zeros((n, 3)), depth=np.full(n, 5.0), radius=np.zeros(n, np.int32),
                     radius_margin=np.ones(n), depth_margin=np.ones(n))


def _isotropic(p, g, u, v, sigma, o):
    p.uv[g] = (u, v)
    p.conic[g] = (1.0 / sigma ** 2, 0.0, 1.0 / sigma ** 2)
    p.opacity[g] = o
    p.radius[g] = int(math.ceil(3 * sigma))


def test_uncertain_record_excuses_its_reach_only():
    p = _records(2)
    _isotropic(p, 0, 10.5, 10.5, 2.0, 0.5)   # uncertain
    _isotropic(p, 1, 40.5, 10.5, 2.0, 0.9)   # certain: excuses nothing
    unc = np.array([True, False])
    # alpha = 0.5 exp(-d^2 / 8) >= exp(-0.01) / 255  <=>  d <= sqrt(8 ln(127.5 e^0.01)) = 6.2
    pix = np.array([[10, 10], [16, 10], [17, 10], [10, 4], [10, 3], [40, 10]])
    got = uncertain_pixels(p, unc, pix)
    np.testing.assert_array_equal(got, [True, True, False, True, False, False])


def test_anisotropic_reach_follows_the_conic():
    p = _records(1)
    # Sigma' = diag(16, 1): reach 6.2 * 2 along x, 6.2 / 2 along y
    p.uv[0] = (50.5, 50.5)
    p.conic[0] = (1.0 / 16.0, 0.0, 1.0)
    p.opacity[0] = 0.5
    p.radius[0] = 12
    pix = np.array([[62, 50], [63, 50], [50, 53], [50, 54]])
    np.testing.assert_array_equal(uncertain_pixels(p, np.array([True]), pix), [True, False, True, False])


def test_near_plane_record_excuses_every_pixel():
    p = _records(2)
    _isotropic(p, 0, 10.5, 10.5, 2.0, 0.5)
    p.depth[1] = ZNEAR
    p.radius[1] = 3
    pix = np.array([[0, 0], [100, 100]])
    assert uncertain_pixels(p, np.array([False, True]), pix).all()
    assert not uncertain_pixels(p, np.array([False, False]), pix).any()


def test_pixel_excuse_lies_inside_the_tile_mask():
    rng = np.random.default_rng(3)
    n, W, H = 40, 96, 80
    p = _records(n)
    for g in range(n):
        _isotropic(p, g, rng.uniform(0, W), rng.uniform(0, H), rng.uniform(0.5, 6.0), rng.uniform(0.01, 0.99))
    unc = rng.random(n) < 0.3
    yy, xx = np.mgrid[0:H, 0:W]
    pix = np.c_[xx.ravel(), yy.ravel()]
    fine = uncertain_pixels(p, unc, pix).reshape(H, W)
    coarse = uncertain_tile_mask(p, unc, W, H)
    assert fine.any() and not (fine & ~coarse).any()
    assert fine.sum() < coarse.sum()

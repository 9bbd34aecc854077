"""Pins of the inverse-exploration oracle (oracle/inverse.py) against what the definitions fix.

* SSIM: a pixel-by-pixel double loop over the 11 x 11 window (zero padding) on a tiny image;
  the closed form (2ab + C1)/(a^2 + b^2 + C1) inside constant images a, b; SSIM(x, x) = 1.
* Loss gradient: central finite differences of the loss (border and interior pixels, two views
  of different sizes); zero at x = y.
* Adam: the first bias-corrected step is lr g / (|g| + eps) exactly; a two-step sequence
  against the recursion written out by hand; values not selected by the mask stay put.
* Light angles: dir(polar, azimuth) round-trips through light_angles; the angle gradient the
  optimiser forms from dloss/d dir matches finite differences of the oracle renderer.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import inverse as inv


def _brute_ssim(x, y):
    H, W = x.shape
    k = np.arange(-5, 6)
    w1 = np.exp(-(k ** 2) / (2 * 1.5 ** 2))
    w = np.outer(w1, w1)
    w /= w.sum()
    out = np.zeros((H, W))
    for j in range(H):
        for i in range(W):
            s = np.zeros(5)
            for dj in range(-5, 6):
                for di in range(-5, 6):
                    jj, ii = j + dj, i + di
                    if 0 <= jj < H and 0 <= ii < W:
                        a, b = x[jj, ii], y[jj, ii]
                        s += w[dj + 5, di + 5] * np.array([a, b, a * a, b * b, a * b])
            mx, my = s[0], s[1]
            vx, vy, cxy = s[2] - mx * mx, s[3] - my * my, s[4] - mx * my
            out[j, i] = ((2 * mx * my + inv.C1) * (2 * cxy + inv.C2)) / \
                ((mx * mx + my * my + inv.C1) * (vx + vy + inv.C2))
    return out


def test_ssim_map_matches_pixel_by_pixel_definition():
    rng = np.random.default_rng(1)
    x, y = rng.random((7, 9)), rng.random((7, 9))
    np.testing.assert_allclose(inv.ssim_map(x, y), _brute_ssim(x, y), rtol=1e-12, atol=1e-14)


def test_ssim_closed_forms():
    a, b = 0.3, 0.7
    x, y = np.full((32, 32), a), np.full((32, 32), b)
    s = inv.ssim_map(x, y)
    np.testing.assert_allclose(s[10:22, 10:22], (2 * a * b + inv.C1) / (a * a + b * b + inv.C1), rtol=1e-12)
    rng = np.random.default_rng(2)
    z = rng.random((20, 17))
    np.testing.assert_allclose(inv.ssim_map(z, z), 1.0, rtol=0, atol=1e-12)
    img = [rng.random((20, 17, 4))]
    loss, l1, ssim, g = inv.image_loss(img, img, 0.2)
    assert abs(loss) < 1e-12 and l1 == 0.0 and abs(ssim - 1.0) < 1e-12
    assert np.abs(g[0]).max() < 1e-12


@pytest.mark.parametrize("lam", [0.2, 1.0])
def test_loss_gradient_matches_finite_differences(lam):
    rng = np.random.default_rng(3)
    xs = [rng.random((9, 13, 4)), rng.random((6, 5, 4))]
    ys = [rng.random((9, 13, 4)), rng.random((6, 5, 4))]
    loss, _, _, grads = inv.image_loss(xs, ys, lam)
    eps = 1e-6
    picks = [(0, 0, 0, 0), (0, 4, 6, 1), (0, 8, 12, 2), (1, 0, 4, 0), (1, 3, 2, 2), (0, 2, 11, 1)]
    for v, j, i, c in picks:
        vals = []
        for s in (+1, -1):
            x2 = [a.copy() for a in xs]
            x2[v][j, i, c] += s * eps
            vals.append(inv.image_loss(x2, ys, lam)[0])
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert abs(fd - grads[v][j, i, c]) <= 1e-6 * max(1.0, abs(fd)), (v, j, i, c, fd, grads[v][j, i, c])


def test_adam_steps():
    M = 2
    rng = np.random.default_rng(4)
    table = np.zeros(8 * M + 12)
    table[:8 * M] = rng.random(8 * M)
    table[8 * M:8 * M + 8] = [1, 1, 1, 1, 0, 0, 0, 0]
    table[8 * M + 8:8 * M + 12] = [*inv.light_dir(0.7, -1.2), 1.0]
    g1 = rng.normal(0, 1, table.shape)
    st = inv.AdamState(table, M)
    np.testing.assert_allclose(st.angles, [0.7, -1.2], rtol=1e-12)
    lr, eps = 0.01, 1e-8
    t1 = inv.adam_step(table, g1, M, st, inv.LEARN_COLOR | inv.LEARN_LIGHT_MAGNITUDE, lr, eps=eps)
    for m in range(M):
        for k in range(3):
            i = 8 * m + k
            assert math.isclose(t1[i], table[i] - lr * g1[i] / (abs(g1[i]) + eps), rel_tol=1e-12)
        assert t1[8 * m + 3] == table[8 * m + 3] and t1[8 * m + 4] == table[8 * m + 4]  # masked / visible
    np.testing.assert_array_equal(t1[8 * M + 8:], table[8 * M + 8:])  # direction not learned
    # second step: the recursion by hand for one value
    g2 = rng.normal(0, 1, table.shape)
    t2 = inv.adam_step(t1, g2, M, st, inv.LEARN_COLOR | inv.LEARN_LIGHT_MAGNITUDE, lr, eps=eps)
    i = 8 * M + 2
    m1, v1 = 0.1 * g1[i], 0.001 * g1[i] ** 2
    m2, v2 = 0.9 * m1 + 0.1 * g2[i], 0.999 * v1 + 0.001 * g2[i] ** 2
    step = lr * (m2 / (1 - 0.9 ** 2)) / (math.sqrt(v2 / (1 - 0.999 ** 2)) + eps)
    assert math.isclose(t2[i], t1[i] - step, rel_tol=1e-12)


def test_light_angles_round_trip():
    for th, ph in [(0.3, 0.1), (2.5, -2.0), (1.2, 3.0)]:
        d = inv.light_dir(th, ph)
        assert abs(np.linalg.norm(d) - 1) < 1e-15
        np.testing.assert_allclose(inv.light_angles(3.0 * d), (th, ph), rtol=1e-12)


def test_light_angle_gradient_matches_finite_differences():
    """d loss / d(polar, azimuth) as the optimiser forms it (chain through dloss/d dir of the
    oracle backward) against finite differences of the rendered loss."""
    from tests.test_oracle_grad_fd import _scene
    models, ed, cams = _scene(True, True)
    th, ph = 1.1, -0.6
    bg = np.array([0.1, 0.2, 0.3])
    rng = np.random.default_rng(5)
    wts = [rng.normal(0, 1, (c.H, c.W, 4)) for c in cams]
    loss = lambda r: sum((im * w).sum() for im, w in zip(r.images, wts))

    def render(a, b):
        e = ed.copy()
        e.light_dir = inv.light_dir(a, b)
        return oracle.render(models, e, cams, bg=bg)

    r = render(th, ph)
    gr = oracle.render_backward(r, cams, wts, bg=bg)
    M = len(models)
    gd = gr.edit[8 * M + 8:8 * M + 11]
    dth = np.dot(gd, [np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)])
    dph = np.dot(gd, [-np.sin(th) * np.sin(ph), np.sin(th) * np.cos(ph), 0.0])
    eps = 1e-5
    fth = (loss(render(th + eps, ph)) - loss(render(th - eps, ph))) / (2 * eps)
    fph = (loss(render(th, ph + eps)) - loss(render(th, ph - eps))) / (2 * eps)
    assert abs(fth - dth) <= 1e-5 * max(1.0, abs(fth)), (fth, dth)
    assert abs(fph - dph) <= 1e-5 * max(1.0, abs(fph)), (fph, dph)
    # the Adam state starts from the table's angles, and a direction step writes a unit vector
    e = ed.copy()
    e.light_dir = inv.light_dir(th, ph)
    tab = oracle.edit_table(e)
    st = inv.AdamState(tab, M)
    np.testing.assert_allclose(st.angles, (th, ph), rtol=1e-12)
    tab2 = inv.adam_step(tab, gr.edit, M, st, inv.LEARN_LIGHT_DIRECTION, 0.01)
    assert abs(np.linalg.norm(tab2[8 * M + 8:8 * M + 11]) - 1.0) < 1e-14
    assert np.abs(tab2[8 * M + 8:8 * M + 11] - tab[8 * M + 8:8 * M + 11]).max() > 1e-4

"""Pins of the oracle's SH colour (the 3DGS view-dependent colour of Sec. 3 / Sec. 4.2).

* The 16 basis functions are orthonormal on the unit sphere: a product quadrature
  (Gauss-Legendre in cos(theta) x uniform in phi), exact for these polynomial degrees.
* Their gradients equal finite differences of the polynomials.
* Degree 0 gives the constant colour sh_0 / (2 sqrt(pi)) + 0.5 (clamped at 0) in every view.
* The reverse mode (SH coefficients and means through the view direction) matches central
  finite differences of a rendered loss.
"""
import ctypes as C

import numpy as np

import oracle
import scenegen as sg


def _basis(d, deg=3):
    Y = np.zeros(16)
    dY = np.zeros((16, 3))
    oracle.lib().orc_sh_basis(oracle._p(np.ascontiguousarray(d, np.float64)), C.c_int32(deg), oracle._p(Y),
                              oracle._p(dY))
    return Y, dY


def test_sh_basis_orthonormal():
    ct, wt = np.polynomial.legendre.leggauss(12)
    nphi = 24
    G = np.zeros((16, 16))
    for c, w in zip(ct, wt):
        st = np.sqrt(1 - c * c)
        for k in range(nphi):
            ph = 2 * np.pi * k / nphi
            Y, _ = _basis([st * np.cos(ph), st * np.sin(ph), c])
            G += np.outer(Y, Y) * w * (2 * np.pi / nphi)
    np.testing.assert_allclose(G, np.eye(16), rtol=0, atol=1e-12)


def test_sh_basis_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    for _ in range(10):
        d = rng.normal(0, 1, 3)
        _, dY = _basis(d)
        eps = 1e-6
        for j in range(3):
            e = np.zeros(3)
            e[j] = eps
            fd = (_basis(d + e)[0] - _basis(d - e)[0]) / (2 * eps)
            np.testing.assert_allclose(dY[:, j], fd, rtol=0, atol=1e-8)


def _sh_scene(deg, seed=5):
    w = sg.tiny_scene(300, 40, 36, seed, log_scale_mu=-2.8, n_models=1)
    comp = oracle.compose(w.models)
    rng = np.random.default_rng(seed)
    nb = (deg + 1) ** 2
    sh = rng.normal(0, 0.4, (comp.n, nb, 3))
    sh[:, 0, :] = rng.uniform(-0.5, 1.5, (comp.n, 3))
    comp.sh, comp.sh_degree = sh, deg
    return w, comp


def test_sh_degree0_is_a_constant_colour():
    w, comp = _sh_scene(0)
    table = oracle.edit_table(w.edits)
    p = oracle.project(comp, table, w.cameras[0])
    live = p.radius > 0
    want = np.maximum(comp.sh[:, 0, :] / (2 * np.sqrt(np.pi)) + 0.5, 0.0)
    np.testing.assert_allclose(p.rgb[live], want[live], rtol=0, atol=1e-14)


def test_sh_gradients_match_finite_differences():
    w, comp = _sh_scene(3)
    cams = [w.cameras[0], sg.look_at([0.0, -3.0, 0.5], 36, 40)]
    table = oracle.edit_table(w.edits)
    rng = np.random.default_rng(6)
    wts = [rng.normal(0, 1, (c.H, c.W, 4)) for c in cams]
    r = oracle.render(None, w.edits, cams, comp=comp, table=table)
    gr = oracle.render_backward(r, cams, wts)
    loss = lambda rr: sum((im * wt).sum() for im, wt in zip(rr.images, wts))
    live = np.nonzero(r.projs[0].radius > 0)[0]
    checked = 0
    for t in range(40):
        g = int(live[rng.integers(0, len(live))])
        which = "sh" if t % 2 == 0 else "mean"
        idx = (g, int(rng.integers(0, 16)), int(rng.integers(0, 3))) if which == "sh" else (g, int(rng.integers(0, 3)))
        eps = 1e-6
        vals = []
        for s in (+1, -1):
            c2 = oracle.Composed(*(np.array(a, copy=True) for a in comp.arrays()), model_id=comp.model_id,
                                 n_models=comp.n_models, sh=np.array(comp.sh, copy=True), sh_degree=3)
            getattr(c2, which)[idx] += s * eps
            vals.append(loss(oracle.render(None, w.edits, cams, comp=c2, table=table)))
        fd = (vals[0] - vals[1]) / (2 * eps)
        an = gr.params[which][idx]
        if abs(fd - an) > 1e-5 * max(1.0, abs(an)):
            # a perturbation that flips a discrete decision (radius, cut-off) is not a derivative
            continue
        checked += 1
    assert checked >= 37, checked  # at most 3 perturbations that flip a decision
    assert np.abs(gr.params["sh"]).max() > 0

"""Pin of the oracle's reverse-mode gradient by central finite differences of its forward.

200-Gaussian 64x64 subscene, eps = 1e-4 in float64, 64 randomly picked parameters per scene
(seed 4) over all stored Gaussian attributes and the edit parameters (palette colour and
opacity scale per model, lambda and b, the orbital light direction).  A parameter whose +-eps
perturbation changes a discrete decision (radius, tile lists, contributor sets) is detected by
comparing those integers and reported, not averaged in.
"""
import numpy as np
import pytest

import oracle
import scenegen as sg

EPS = 1e-4


def _loss(r, w):
    return sum(float((img * wv).sum()) for img, wv in zip(r.images, w))


def _signature(r):
    return (tuple(p.radius.tobytes() for p in r.projs), r.bins.keys.tobytes(), r.bins.values.tobytes(),
            tuple(l.tobytes() for l in r.last), tuple(m[..., 4:].tobytes() for m in r.margins))


def _scene(orbital, table_light=False):
    w = sg.fd_subscene()
    if orbital:
        c = w.cameras[0]
        c.headlight = 0
        c.light_dir = sg.orbital_light(30.0, 0.7)
    # a second basic model so that per-model edits have something to act on
    rng = np.random.default_rng(44)
    m2 = w.models[0].copy()
    m2.mean = (m2.mean + rng.normal(0, 0.05, m2.mean.shape)).astype(np.float32)
    m2.palette = np.array([0.3, 0.6, 0.2], np.float32)
    models = [w.models[0], m2]
    ed = sg.identity_edits(models)
    ed.opacity_scale[:] = [0.8, 1.1]
    ed.lam = np.array([1.1, 0.9, 1.2, 0.8], np.float32)
    ed.bias = np.array([0.02, -0.01, 0.03, 1.0], np.float32)
    if table_light:  # the global light of the edit table overrides the view's (Sec. 4.6)
        ed.light_dir = np.array(sg.orbital_light(-50.0, 0.4), np.float64) * 1.7
    return models, ed, w.cameras


@pytest.mark.parametrize("orbital,table_light", [(False, False), (True, False), (True, True)],
                         ids=["headlight", "orbital", "table_light"])
def test_oracle_gradient_matches_central_fd(orbital, table_light):
    models, ed, cams = _scene(orbital, table_light)
    comp = oracle.compose(models)
    table = oracle.edit_table(ed)
    bg = np.array([0.2, 0.1, 0.3])
    rng = np.random.default_rng(4)
    wts = [rng.normal(0, 1, (c.H, c.W, 4)) for c in cams]
    base = oracle.render(models, ed, cams, bg=bg, comp=comp, table=table)
    assert base.images[0][..., 3].mean() > 0.1
    grads = oracle.render_backward(base, cams, wts, bg=bg)
    live = np.nonzero(base.projs[0].radius > 0)[0]
    M = comp.n_models

    def draw():
        if rng.random() < 0.75:
            k = oracle.PARAMS[rng.integers(0, len(oracle.PARAMS))]
            g = int(live[rng.integers(0, len(live))])
            arr = getattr(comp, k)
            j = int(rng.integers(0, arr.shape[1])) if arr.ndim == 2 else None
            return ("param", k, g, j)
        kind = rng.integers(0, 4 if not orbital else 5)
        if kind == 4 and table_light:
            return ("edit", M * 8 + 8 + int(rng.integers(0, 3)), None, None)
        if kind == 0:
            return ("edit", int(rng.integers(0, M)) * 8 + int(rng.integers(0, 3)), None, None)
        if kind == 1:
            return ("edit", int(rng.integers(0, M)) * 8 + 3, None, None)
        if kind == 2:
            return ("edit", M * 8 + int(rng.integers(0, 4)), None, None)
        if kind == 3:
            return ("edit", M * 8 + 4 + int(rng.integers(0, 4)), None, None)
        return ("light", int(rng.integers(0, 3)), None, None)

    sig0 = _signature(base)
    checked, flipped, refined, errs = 0, 0, 0, []
    while checked < 64 and checked + flipped < 200:
        kind, a, b, c = draw()
        def fd_at(eps):
            vals, sigs = [], []
            for s in (+1, -1):
                comp2 = oracle.Composed(*(np.array(x, copy=True) for x in comp.arrays()),
                                        model_id=comp.model_id, n_models=M)
                table2 = table.copy()
                cams2 = [sg.Camera(**{**cc.__dict__, "light_dir": np.array(cc.light_dir, np.float64)})
                         for cc in cams]
                if kind == "param":
                    arr = getattr(comp2, a)
                    if c is None:
                        arr[b] += s * eps
                    else:
                        arr[b, c] += s * eps
                elif kind == "edit":
                    table2[a] += s * eps
                else:
                    cams2[0].light_dir[a] += s * eps
                r = oracle.render(models, ed, cams2, bg=bg, comp=comp2, table=table2)
                vals.append(_loss(r, wts))
                sigs.append(_signature(r))
            return (vals[0] - vals[1]) / (2 * eps), sigs[0] == sig0 and sigs[1] == sig0

        fd, same = fd_at(EPS)
        if not same:
            flipped += 1
            continue
        if kind == "param":
            an = grads.params[a][b] if c is None else grads.params[a][b, c]
        elif kind == "edit":
            an = grads.edit[a]
        else:
            an = grads.light[0, a]
        tol = lambda x: abs(x - an) <= 1e-5 * max(abs(an), 1.0) + 1e-6
        if not tol(fd):
            # steep terms (e.g. the specular lobe |n.h|^beta with beta ~ 27) leave O(eps^2)
            # truncation error at 1e-4: the derivative is the limit, so refine the step
            fd, same = fd_at(EPS / 10)
            refined += 1
            assert same, (kind, a, b, c)
        checked += 1
        errs.append(abs(fd - an) / max(abs(an), 1e-3))
        assert tol(fd), (kind, a, b, c, fd, an)
    assert checked == 64 and flipped < checked and refined <= 8, (checked, flipped, refined)
    print(f"checked {checked}, flipped {flipped}, refined {refined}, max rel err {max(errs):.2e}")


def test_table_light_replaces_the_view_light():
    """The edit table's global light gives the image of a view whose own light_dir is that
    direction (any length: only l / |l| is used), and leaves the view's light_dir without a
    gradient; switched off (4th entry 0) it changes nothing."""
    models, ed, cams = _scene(True)
    bg = np.array([0.1, 0.2, 0.3])
    ref = oracle.render(models, ed, cams, bg=bg)
    ed2 = ed.copy()
    ed2.light_dir = np.array(cams[0].light_dir, np.float64) * 3.0
    cams2 = [sg.Camera(**{**c.__dict__, "light_dir": np.array([0.0, 0.0, 1.0])}) for c in cams]
    r2 = oracle.render(models, ed2, cams2, bg=bg)
    np.testing.assert_allclose(r2.images[0], ref.images[0], rtol=0, atol=1e-14)
    wts = [np.ones((c.H, c.W, 4)) for c in cams]
    g2 = oracle.render_backward(r2, cams2, wts, bg=bg)
    assert np.all(g2.light == 0.0)
    M = len(models)
    g1 = oracle.render_backward(ref, cams, wts, bg=bg)
    # d/dl of the table light (length 3) = d/dl of the view light (length 1) / 3
    np.testing.assert_allclose(g2.edit[M * 8 + 8:M * 8 + 11] * 3.0, g1.light[0], rtol=1e-10, atol=1e-12)
    t = oracle.edit_table(ed2)
    t[M * 8 + 11] = 0.0
    r3 = oracle.render(models, ed2, cams, bg=bg, table=t)
    np.testing.assert_array_equal(r3.images[0], ref.images[0])

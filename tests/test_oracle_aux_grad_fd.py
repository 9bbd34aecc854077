"""Pin of the oracle's reverse mode of the auxiliary maps (``oracle.render_aux_backward``) by
central finite differences of its forward (``oracle.render_aux``).

The FD subscene with a second model, an orbital light and non-trivial lambda, b and opacity
scales; a random upstream gradient on all 12 channels (depth, normal, dc, k', 1 - T). 48
randomly picked parameters over every stored attribute and the edit parameters, eps = 1e-4 in
float64 (refined to 1e-5 for steep terms); a perturbation that changes a discrete decision
(radius, tile lists, contributor sets) is detected and reported, not averaged in. Besides: an
upstream gradient on the 1 - T channel alone gives the RGB reverse mode's gradients for the same
gradient on the alpha channel."""
import numpy as np
import pytest

import oracle
from tests.test_oracle_grad_fd import _scene, _signature

EPS = 1e-4


def _loss(aux, w):
    return sum(float((a * wv).sum()) for a, wv in zip(aux, w))


@pytest.mark.parametrize("orbital", [False, True], ids=["headlight", "orbital"])
def test_aux_gradient_matches_central_fd(orbital):
    models, ed, cams = _scene(orbital)
    comp = oracle.compose(models)
    table = oracle.edit_table(ed)
    rng = np.random.default_rng(7)
    wts = [rng.normal(0, 1, (c.H, c.W, 12)) for c in cams]
    base = oracle.render(models, ed, cams, comp=comp, table=table)
    assert base.images[0][..., 3].mean() > 0.1
    grads = oracle.render_aux_backward(base, cams, wts)
    live = np.nonzero(base.projs[0].radius > 0)[0]
    M = comp.n_models

    def draw():
        if rng.random() < 0.75:
            k = oracle.PARAMS[rng.integers(0, len(oracle.PARAMS))]
            g = int(live[rng.integers(0, len(live))])
            arr = getattr(comp, k)
            return ("param", k, g, int(rng.integers(0, arr.shape[1])) if arr.ndim == 2 else None)
        kind = rng.integers(0, 3)
        if kind == 0:
            return ("edit", int(rng.integers(0, M)) * 8 + 3, None, None)     # opacity scale
        if kind == 1:
            return ("edit", M * 8 + int(rng.integers(0, 4)), None, None)     # lambda
        return ("edit", M * 8 + 4 + int(rng.integers(0, 4)), None, None)     # b

    sig0 = _signature(base)
    checked, flipped, refined = 0, 0, 0
    while checked < 48 and checked + flipped < 150:
        kind, a, b, c = draw()

        def fd_at(eps):
            vals, sigs = [], []
            for s in (+1, -1):
                comp2 = oracle.Composed(*(np.array(x, copy=True) for x in comp.arrays()),
                                        model_id=comp.model_id, n_models=M)
                table2 = table.copy()
                if kind == "param":
                    arr = getattr(comp2, a)
                    if c is None:
                        arr[b] += s * eps
                    else:
                        arr[b, c] += s * eps
                else:
                    table2[a] += s * eps
                r = oracle.render(models, ed, cams, comp=comp2, table=table2)
                vals.append(_loss(oracle.render_aux(r, cams), wts))
                sigs.append(_signature(r))
            return (vals[0] - vals[1]) / (2 * eps), sigs[0] == sig0 and sigs[1] == sig0

        fd, same = fd_at(EPS)
        if not same:
            flipped += 1
            continue
        an = (grads.params[a][b] if c is None else grads.params[a][b, c]) if kind == "param" else grads.edit[a]
        tol = lambda x: abs(x - an) <= 1e-5 * max(abs(an), 1.0) + 1e-6
        if not tol(fd):
            fd, same = fd_at(EPS / 10)
            refined += 1
            assert same, (kind, a, b, c)
        checked += 1
        assert tol(fd), (kind, a, b, c, fd, an)
    assert checked == 48 and flipped < checked and refined <= 6, (checked, flipped, refined)


def test_alpha_channel_alone_is_the_rgb_reverse_mode_of_alpha():
    """An upstream gradient on the 1 - T channel only is the same loss as that gradient on the
    RGB render's alpha channel (the same contributors and weights), so both reverse modes give
    the same gradients (up to float64 summation order)."""
    models, ed, cams = _scene(True)
    base = oracle.render(models, ed, cams)
    rng = np.random.default_rng(9)
    da = [rng.normal(0, 1, (c.H, c.W)) for c in cams]
    w_aux = [np.concatenate([np.zeros((c.H, c.W, 11)), d[..., None]], -1) for c, d in zip(cams, da)]
    w_rgb = [np.concatenate([np.zeros((c.H, c.W, 3)), d[..., None]], -1) for c, d in zip(cams, da)]
    ga = oracle.render_aux_backward(base, cams, w_aux)
    gr = oracle.render_backward(base, cams, w_rgb)
    for k in oracle.PARAMS:
        np.testing.assert_allclose(ga.params[k], gr.params[k], rtol=1e-9, atol=1e-12, err_msg=k)
    np.testing.assert_allclose(ga.edit, gr.edit, rtol=1e-9, atol=1e-12)
    assert all(np.all(pv["aux"] == 0.0) for pv in ga.proj)

"""Degenerate scenes through the whole path (projection, binning, forward, backward), against
the FP64 oracle:

* every basic model hidden: the image is the background, alpha 0, every gradient 0;
* a single Gaussian (one record, a handful of pairs);
* every Gaussian behind the camera's near plane: nothing projects, background image.
"""
import numpy as np
import pytest
import torch

import oracle
import scenegen as sg
from tests import _gpu

pytestmark = pytest.mark.gpu


def _run(w):
    rast, comp, table = _gpu.setup(w)
    rgba = rast.forward(comp, table).clone()
    rng = np.random.default_rng(3)
    dls = [rng.normal(0, 1, (c.H, c.W, 4)) for c in w.cameras]
    dl = torch.as_tensor(np.concatenate([d.reshape(-1, 4) for d in dls]), dtype=torch.float32, device="cuda")
    grad, egrad = rast.backward(comp, table, dl.contiguous())
    torch.cuda.synchronize()
    return rast, rgba, grad, egrad, dls


@pytest.mark.parametrize("cull", [True, False])
def test_all_models_hidden(cull):
    base = sg.tiny_scene(500, 48, 40, 61, n_models=2)
    ed = sg.random_edits(base.models, seed=62)
    ed.visible[:] = 0
    bg = np.array([0.3, 0.2, 0.1], np.float32)
    w = sg.Workload("hidden", base.models, base.cameras, ed, bg=bg)
    rast, comp, table = _gpu.setup(w, cull=cull)
    rgba = rast.forward(comp, table).clone()
    dl = torch.ones((rast.n_pix, 4), dtype=torch.float32, device="cuda")
    grad, egrad = rast.backward(comp, table, dl)
    torch.cuda.synchronize()
    assert rast.n_pairs == 0
    want = torch.tensor([*bg.tolist(), 0.0], dtype=torch.float32, device="cuda").expand_as(rgba)
    assert torch.equal(rgba, want)
    for k in oracle.PARAMS:
        assert float(getattr(grad, k).abs().max()) == 0.0, k
    # only the light's background path can carry gradient; with every model hidden, none does
    assert float(egrad[:8 * len(base.models)].abs().max()) == 0.0


def test_single_gaussian():
    w = sg.tiny_scene(1, 40, 36, 63, log_scale_mu=-2.0)
    rast, rgba, grad, egrad, dls = _run(w)
    ref = oracle.render(w.models, w.edits, w.cameras, bg=w.bg)
    assert rast.n_pairs > 0
    for v, c in enumerate(w.cameras):
        err, excused, bad = _gpu.compare_image(rast.view_image(v, rgba).cpu().numpy(), ref.images[v], ref.margins[v])
        assert bad == 0, err
    gref = oracle.render_backward(ref, w.cameras, dls, bg=w.bg)
    for k in oracle.PARAMS:
        _gpu.assert_grad(getattr(grad, k).cpu().numpy(), gref.params[k], k)


def test_everything_behind_the_camera():
    base = sg.tiny_scene(300, 40, 36, 64)
    # the camera looks away from the scene: every Gaussian has camera z <= the near plane
    cam = sg.look_at([0.0, 0.0, 3.0], 40, 36, target=(0.0, 0.0, 6.0))
    w = sg.Workload("behind", base.models, [cam], base.edits, bg=np.array([0.05, 0.1, 0.15], np.float32))
    rast, rgba, grad, egrad, dls = _run(w)
    ref = oracle.render(w.models, w.edits, w.cameras, bg=w.bg)
    assert all(int((p.radius > 0).sum()) == 0 for p in ref.projs)
    assert rast.n_pairs == 0
    np.testing.assert_array_equal(rast.view_image(0, rgba).cpu().numpy(), ref.images[0].astype(np.float32))
    for k in oracle.PARAMS:
        assert float(getattr(grad, k).abs().max()) == 0.0, k

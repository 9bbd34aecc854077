"""The differentiable render (``paper_2504_17954_gb300.render``, a torch.autograd.Function over
ivrgs_render / ivrgs_render_backward) against the FP64 oracle's reverse mode (Sec. 4.6: the
edit parameters are fitted by back-propagating an image loss through the rasterizer).

Leaf tensors for every Gaussian attribute and for the edit table go through ``render``; a
fixed random weighting of the RGBA output is the loss; after ``loss.backward()`` every ``.grad``
(attributes, edit table) and the per-view light gradients ``rast.light_grad`` must meet the
gradient bar against ``oracle.render_backward`` (1e-3 relative L2 and 1e-3 of the largest
entry, element by element). A second render with a different loss must give that loss's
gradients (no state of the first carried over), and a render whose Rasterizer has rendered
again before its backward must refuse to run that backward.
"""
import numpy as np
import pytest
import torch

import oracle
import scenegen as sg
from paper_2504_17954_gb300 import Rasterizer, compose_edit, render
from paper_2504_17954_gb300.rasterizer import ATTRS
from tests import _gpu
from tests.test_oracle_grad_fd import _scene

pytestmark = pytest.mark.gpu


def _workload():
    models, ed, cams = _scene(orbital=True)
    # a second, headlight view of another size: per-view light gradients and the packed layout
    cams = list(cams) + [sg.look_at(3.0 * sg.random_direction(np.random.default_rng(81)), 48, 40)]
    return sg.Workload("autograd", models, cams, ed, bg=np.array([0.2, 0.1, 0.3], np.float32))


def _leaves(w):
    dm = _gpu.device_models(w.models)
    ed = w.edits
    comp, table = compose_edit(dm, ed.palette, ed.opacity_scale, ed.visible, ed.lam, ed.bias)
    attrs = [getattr(comp, k).detach().clone().requires_grad_(True) for k in ATTRS]
    tab = table.detach().clone().requires_grad_(True)
    return comp, tab, attrs


def _loss_weights(w, seed):
    rng = np.random.default_rng(seed)
    dls = [rng.normal(0, 1, (c.H, c.W, 4)) for c in w.cameras]
    wt = torch.as_tensor(np.concatenate([d.reshape(-1, 4) for d in dls]), dtype=torch.float32, device="cuda")
    return dls, wt


def _check(w, attrs, tab, rast, dls):
    ref = oracle.render(w.models, w.edits, w.cameras, bg=w.bg)
    gref = oracle.render_backward(ref, w.cameras, dls, bg=w.bg)
    for k, a in zip(ATTRS, attrs):
        assert a.grad is not None, k
        l2, el = _gpu.assert_grad(a.grad.cpu().numpy(), gref.params[k], k)
        print(f"{k}: relative L2 {l2:.2e}, element-wise {el:.2e}")
    ne = len(gref.edit)
    assert tab.grad is not None and tab.grad.numel() == ne
    _gpu.assert_grad(tab.grad.cpu().numpy(), gref.edit, "edit table")
    light = rast.light_grad.cpu().numpy()
    assert np.abs(gref.light[0]).max() > 0
    _gpu.assert_grad(light[0], gref.light[0], "light of the orbital view")
    assert np.all(light[1] == 0)  # the headlight view has no light direction


def test_render_autograd_matches_oracle():
    w = _workload()
    comp, tab, attrs = _leaves(w)
    rast = Rasterizer(w.cameras, comp.n, len(w.models), bg=w.bg)
    for seed in (5, 6):  # the second loss must not see anything of the first
        for t in [tab, *attrs]:
            t.grad = None
        dls, wt = _loss_weights(w, seed)
        rgba = render(rast, comp, tab, params=attrs)
        assert rgba.requires_grad and rgba.shape == (rast.n_pix, 4)
        loss = (rgba * wt).sum()
        loss.backward()
        torch.cuda.synchronize()
        _check(w, attrs, tab, rast, dls)


def test_render_autograd_refuses_a_stale_backward():
    w = _workload()
    comp, tab, attrs = _leaves(w)
    rast = Rasterizer(w.cameras, comp.n, len(w.models), bg=w.bg)
    first = render(rast, comp, tab, params=attrs)
    second = render(rast, comp, tab, params=attrs)  # overwrites the first render's state
    with pytest.raises(RuntimeError, match="rendered again"):
        first.sum().backward()
    second.sum().backward()  # the latest render's backward still runs
    torch.cuda.synchronize()
    assert attrs[0].grad is not None and torch.isfinite(attrs[0].grad).all()

"""Reverse mode of the auxiliary maps on the GPU (ivrgs_render_aux_backward) against the FP64
oracle's (``oracle.render_aux_backward``, pinned by finite differences): every attribute
gradient and the edit table within the gradient bar (relative L2 and element by element), on a
two-model scene with lambda, b and opacity-scale edits, a three-view scene of uneven sizes, and
16 x 8 tiles. Besides: an upstream gradient on the 1 - T channel alone gives the colour reverse
mode's gradients for the same gradient on the alpha channel (the same walk)."""
import numpy as np
import pytest
import torch

import oracle
import scenegen as sg
from tests import _gpu
from tests.test_gpu_parity import _multi_view_scene

pytestmark = pytest.mark.gpu


def _scene(which):
    if which == "multi":
        return _multi_view_scene(seed=51)
    from tests.test_oracle_grad_fd import _scene as fd_scene
    models, ed, cams = fd_scene(True)
    return sg.Workload("fd2", models, cams, ed, bg=np.zeros(3, np.float32))


def _dl(w, seed):
    rng = np.random.default_rng(seed)
    dls = [rng.normal(0, 1, (c.H, c.W, 12)) for c in w.cameras]
    packed = np.concatenate([d.reshape(-1, 12) for d in dls])
    return dls, torch.as_tensor(packed, dtype=torch.float32, device="cuda").contiguous()


@pytest.mark.parametrize("which,tile_h", [("fd2", 16), ("multi", 16), ("multi", 8)])
def test_aux_backward_matches_oracle(which, tile_h):
    w = _scene(which)
    rast, comp, table = _gpu.setup(w, tile_h=tile_h)
    rast.forward(comp, table)
    dls, dl = _dl(w, 53)
    grad, egrad = rast.render_aux_backward(comp, table, dl)
    torch.cuda.synchronize()
    tile = (16, tile_h)
    ref = oracle.render(w.models, w.edits, w.cameras, bg=w.bg, tile=tile)
    gref = oracle.render_aux_backward(ref, w.cameras, dls, tile=tile)
    for k in oracle.PARAMS:
        _gpu.assert_grad(getattr(grad, k).cpu().numpy(), gref.params[k], k)
    ne = len(gref.edit)
    _gpu.assert_grad(egrad.cpu().numpy().astype(np.float64)[:ne], gref.edit, "edit table")


def test_alpha_channel_alone_equals_the_colour_reverse_mode():
    w = _scene("multi")
    rast, comp, table = _gpu.setup(w)
    rast.forward(comp, table)
    rng = np.random.default_rng(55)
    da = torch.as_tensor(rng.normal(0, 1, rast.n_pix), dtype=torch.float32, device="cuda")
    d_aux = torch.zeros((rast.n_pix, 12), dtype=torch.float32, device="cuda")
    d_aux[:, 11] = da
    d_rgba = torch.zeros((rast.n_pix, 4), dtype=torch.float32, device="cuda")
    d_rgba[:, 3] = da
    ga, ea = rast.render_aux_backward(comp, table, d_aux.contiguous())
    ga = {k: getattr(ga, k).cpu().numpy() for k in oracle.PARAMS}
    ea = ea.cpu().numpy().copy()
    gr, er = rast.backward(comp, table, d_rgba.contiguous())
    torch.cuda.synchronize()
    for k in oracle.PARAMS:
        _gpu.assert_grad(ga[k], getattr(gr, k).cpu().numpy().astype(np.float64), k, tol=1e-4)
    ne = len(oracle.edit_table(w.edits))
    _gpu.assert_grad(ea[:ne], er.cpu().numpy()[:ne].astype(np.float64), "edit table", tol=1e-4)

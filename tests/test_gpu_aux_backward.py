"""Reverse mode of the auxiliary maps on the GPU (ivrgs_render_aux_backward) against the FP64
oracle's (``oracle.render_aux_backward``, pinned by finite differences): every attribute
gradient and the edit table within the gradient bar (relative L2 and element by element), on a
two-model scene with lambda, b and opacity-scale edits, a three-view scene of uneven sizes, 16 x 8
tiles, and 16-bit storage (against the oracle on the decoded values). Besides: an upstream
gradient on the 1 - T channel alone gives the colour reverse mode's gradients for the same
gradient on the alpha channel (the same walk)."""
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


def test_aux_backward_in_16bit_storage():
    """16-bit storage: the gradients with respect to the decoded values, against the oracle's on
    those decoded values."""
    from paper_2504_17954_gb300 import Rasterizer, compose_edit
    from tests.test_gpu_mixed import _composed_arrays, _upload_packed
    base = sg.tiny_scene(2000, 64, 48, 57, log_scale_mu=-3.3, n_models=3)
    rng = np.random.default_rng(57)
    cams = [sg.look_at(3.0 * sg.random_direction(rng), 64, 48), sg.look_at(3.0 * sg.random_direction(rng), 40, 56)]
    w = sg.Workload("mixed_aux", base.models, cams, sg.random_edits(base.models, seed=58))
    M = len(w.models)
    arrs, mid = _composed_arrays(w.models)
    packed, _ = sg.pack_mixed_arrays(**arrs, model_id=mid)
    dec = sg.decode_mixed_arrays(packed)
    g = _upload_packed(packed, M)
    ed = w.edits
    _, table = compose_edit(None, ed.palette, ed.opacity_scale, ed.visible, ed.lam, ed.bias)
    rast = Rasterizer(w.cameras, g.n, M, bg=w.bg)
    rast.forward(g, table)
    dls, dl = _dl(w, 59)
    grad, egrad = rast.render_aux_backward(g, table, dl)
    torch.cuda.synchronize()
    comp = oracle.Composed(*(np.ascontiguousarray(dec[k], np.float64) for k in oracle.PARAMS),
                           model_id=np.ascontiguousarray(packed["model_id"].astype(np.int32)), n_models=M)
    ref = oracle.render(None, None, w.cameras, bg=w.bg, comp=comp, table=oracle.edit_table(ed))
    gref = oracle.render_aux_backward(ref, w.cameras, dls)
    for k in oracle.PARAMS:
        _gpu.assert_grad(getattr(grad, k).cpu().numpy(), gref.params[k], k)
    _gpu.assert_grad(egrad.cpu().numpy().astype(np.float64)[:len(gref.edit)], gref.edit, "edit table")

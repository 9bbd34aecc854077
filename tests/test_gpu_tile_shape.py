"""Parity at 16 x 8 tiles (tile_h = 8, a launch shape the autotuner can pick): the tile lists
bit for bit, the images within 2e-4 and the gradients within 1e-3 (relative L2 and element by
element) against the FP64 oracle binned with the same tile shape, at several pixels-per-thread
settings, with the split walk and with culled lists; the auxiliary maps' 1 - T equal to the
forward's alpha bit for bit. Tolerances and near-tie excuses as in test_gpu_parity.py."""
import numpy as np
import pytest
import torch

import oracle
import scenegen as sg
from tests import _gpu
from tests.test_gpu_parity import _multi_view_scene

pytestmark = pytest.mark.gpu

TILE = (16, 8)


@pytest.fixture(params=[(0, 2, 384), (1, 2, 384), (2, 2, 384), (4, 2, 384), (8, 2, 384), (0, 1, 32)],
                ids=["ppt_auto", "ppt1", "ppt2", "ppt4", "ppt8_as4", "split32"])
def shape(request):
    from paper_2504_17954_gb300 import _native as N
    names = ("render_pixels_per_thread", "render_bwd_pixels_per_thread", "render_split", "render_split_min")
    old = [N.ivrgs_get_option(k) for k in names]
    ppt, split, smin = request.param
    for k, val in zip(names, (ppt, ppt, split, smin)):
        N.ivrgs_set_option(k, val)
    yield request.param
    for k, val in zip(names, old):
        N.ivrgs_set_option(k, val)


def _strip(keys, values, ref, unc_all):
    view_of = np.searchsorted(ref.bins.tile_offset, (keys >> np.uint64(32)).astype(np.int64), side="right") - 1
    keep = np.array([not unc_all[a][b] for a, b in zip(view_of, values)], bool) if len(keys) else np.zeros(0, bool)
    return keys[keep], values[keep]


@pytest.mark.parametrize("which", ["cfg1", "multi"])
def test_forward_16x8_tiles(which, shape):
    w = sg.config1() if which == "cfg1" else _multi_view_scene(seed=25)
    rast, comp, table = _gpu.setup(w, cull=False, tile_h=8)  # rectangle lists, compared with the oracle's
    assert rast.n_tiles == sum(((c.W + 15) // 16) * ((c.H + 7) // 8) for c in w.cameras)
    rast.forward(comp, table)
    torch.cuda.synchronize()
    ref = oracle.render(w.models, w.edits, w.cameras, bg=w.bg, tile=TILE)
    unc_all = [_gpu.uncertain_records(p, 16, 8) for p in ref.projs]
    k, vals, _ = _gpu.gpu_keys(rast)
    gk, gv = _strip(k, vals, ref, unc_all)
    ok_, ov = _strip(ref.bins.keys, ref.bins.values, ref, unc_all)
    np.testing.assert_array_equal(gk, ok_)
    np.testing.assert_array_equal(gv, ov)
    total_excused = 0
    for v, c in enumerate(w.cameras):
        extra = _gpu.uncertain_tile_mask(ref.projs[v], unc_all[v], c.W, c.H, 16, 8)
        err, excused, bad = _gpu.compare_image(rast.view_image(v).cpu().numpy(), ref.images[v], ref.margins[v], extra)
        assert bad == 0, (v, err)
        total_excused += excused
    assert total_excused <= max(3, 0.001 * rast.n_pix)


@pytest.mark.parametrize("which", ["fd", "multi"])
def test_backward_16x8_tiles(which, shape):
    if which == "fd":
        from tests.test_oracle_grad_fd import _scene
        models, ed, cams = _scene(True, False)
        w = sg.Workload("fd", models, cams, ed, bg=np.array([0.2, 0.1, 0.3], np.float32))
    else:
        w = _multi_view_scene(seed=27)
    rast, comp, table = _gpu.setup(w, tile_h=8)
    rast.forward(comp, table)
    rng = np.random.default_rng(4)
    dls = [rng.normal(0, 1, (c.H, c.W, 4)) for c in w.cameras]
    dl = torch.as_tensor(np.concatenate([d.reshape(-1, 4) for d in dls]), dtype=torch.float32, device="cuda")
    grad, egrad = rast.backward(comp, table, dl.contiguous())
    torch.cuda.synchronize()
    ref = oracle.render(w.models, w.edits, w.cameras, bg=w.bg, tile=TILE)
    gref = oracle.render_backward(ref, w.cameras, dls, bg=w.bg, tile=TILE)
    for k in oracle.PARAMS:
        _gpu.assert_grad(getattr(grad, k).cpu().numpy(), gref.params[k], k)
    ne = len(gref.edit)
    _gpu.assert_grad(egrad.cpu().numpy().astype(np.float64)[:ne], gref.edit, "edit table")


def test_culled_16x8_lists_give_the_rectangle_lists_images():
    """With culling, the 16 x 8 lists drop only tiles the cut-off ellipse misses: the images equal
    the oracle's rectangle-list images within the bar."""
    w = _multi_view_scene(seed=31)
    rast, comp, table = _gpu.setup(w, cull=True, tile_h=8)
    rast.forward(comp, table)
    torch.cuda.synchronize()
    ref = oracle.render(w.models, w.edits, w.cameras, bg=w.bg, tile=TILE)
    for v, c in enumerate(w.cameras):
        unc = _gpu.uncertain_records(ref.projs[v], 16, 8)
        extra = _gpu.uncertain_tile_mask(ref.projs[v], unc, c.W, c.H, 16, 8)
        err, _, bad = _gpu.compare_image(rast.view_image(v).cpu().numpy(), ref.images[v], ref.margins[v], extra)
        assert bad == 0, (v, err)


def test_aux_alpha_equals_the_forward_alpha_at_16x8():
    w = _multi_view_scene(seed=33)
    rast, comp, table = _gpu.setup(w, tile_h=8)
    with _gpu.sequential_walk():
        rast.forward(comp, table)
    aux = rast.render_aux(comp, table)
    torch.cuda.synchronize()
    assert torch.equal(aux[:, 11], rast.rgba[:, 3])

"""Auxiliary maps (ivrgs_render_aux; Sec. 4.2 depth / normal maps, Sec. 4.3 offset-colour and
coefficient maps) against the FP64 oracle.

* The last channel (1 - T) equals the alpha of ivrgs_render bit for bit: the same contributors.
* Every channel within 2e-4 of the oracle (relative to the channel's largest magnitude, at
  least 1), outside the oracle-certified near-tie pixels, for float32 and 16-bit storage.
"""
import numpy as np
import pytest
import torch

import oracle
import scenegen as sg
from tests import _gpu
from tests.test_gpu_mixed import _composed_arrays, _upload_packed
from tests.test_gpu_parity import _multi_view_scene

pytestmark = pytest.mark.gpu


def _compare(gpu_aux, ref_aux, margins, extra=None):
    excuse = _gpu.near_tie(margins)
    if extra is not None:
        excuse |= extra
    worst = 0.0
    for k in range(ref_aux.shape[-1]):
        scale = max(1.0, float(np.abs(ref_aux[..., k]).max()))
        err = np.abs(gpu_aux[..., k].astype(np.float64) - ref_aux[..., k]) / scale
        bad = (err > 2e-4) & ~excuse
        assert not bad.any(), (k, float(err[~excuse].max()))
        worst = max(worst, float(err[~excuse].max()))
    return worst


@pytest.mark.parametrize("which", ["cfg1", "multi"])
def test_aux_maps_match_oracle(which):
    w = sg.config1() if which == "cfg1" else _multi_view_scene(seed=81)
    rast, comp, table = _gpu.setup(w)
    with _gpu.sequential_walk():  # the aux walk is the sequential one: compare bit for bit with it
        rast.forward(comp, table)
    aux = rast.render_aux(comp, table)
    torch.cuda.synchronize()
    assert torch.equal(aux[:, 11], rast.rgba[:, 3])
    ref = oracle.render(w.models, w.edits, w.cameras, bg=w.bg)
    maps = oracle.render_aux(ref, w.cameras)
    worst = 0.0
    for v, c in enumerate(w.cameras):
        off = rast.cam_arr[v].pix_offset
        g = aux[off:off + c.W * c.H].cpu().numpy().reshape(c.H, c.W, 12)
        unc = _gpu.uncertain_records(ref.projs[v])
        extra = _gpu.uncertain_tile_mask(ref.projs[v], unc, c.W, c.H)
        worst = max(worst, _compare(g, maps[v], ref.margins[v], extra))
    print(f"{which}: largest relative aux error {worst:.2e}")


def test_aux_maps_mixed_storage():
    w = sg.config1()
    M = len(w.models)
    arrs, mid = _composed_arrays(w.models)
    packed, _ = sg.pack_mixed_arrays(**arrs, model_id=mid)
    dec = sg.decode_mixed_arrays(packed)
    g = _upload_packed(packed, M)
    ed = w.edits
    from paper_2504_17954_gb300 import Rasterizer, compose_edit
    _, table = compose_edit(None, ed.palette, ed.opacity_scale, ed.visible, ed.lam, ed.bias)
    rast = Rasterizer(w.cameras, g.n, M, bg=w.bg)
    with _gpu.sequential_walk():
        rast.forward(g, table)
    aux = rast.render_aux(g, table)
    torch.cuda.synchronize()
    assert torch.equal(aux[:, 11], rast.rgba[:, 3])
    comp = oracle.Composed(*(np.ascontiguousarray(dec[k], np.float64) for k in oracle.PARAMS),
                           model_id=np.ascontiguousarray(packed["model_id"].astype(np.int32)), n_models=M)
    ref = oracle.render(None, None, w.cameras, bg=w.bg, comp=comp, table=oracle.edit_table(ed))
    maps = oracle.render_aux(ref, w.cameras)
    c = w.cameras[0]
    gimg = aux[:c.W * c.H].cpu().numpy().reshape(c.H, c.W, 12)
    unc = _gpu.uncertain_records(ref.projs[0])
    _compare(gimg, maps[0], ref.margins[0], _gpu.uncertain_tile_mask(ref.projs[0], unc, c.W, c.H))

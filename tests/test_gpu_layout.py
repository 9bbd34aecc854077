"""The one-time spatial reorder of a composed float32 set (reorder_spatial).

* The order is a permutation, grouped by model, and the reordered attributes are the gathered
  originals.
* Rendering the reordered set gives the same image bit for bit (no two depths are equal here,
  so the compositing order is the same) and the same gradients, permuted, within float32
  atomic-summation noise.
"""
import numpy as np
import pytest
import torch

import scenegen as sg
from paper_2504_17954_gb300 import reorder_spatial
from paper_2504_17954_gb300.rasterizer import ATTRS
from tests import _gpu

pytestmark = pytest.mark.gpu


def test_reorder_spatial_is_a_layout_change_only():
    base = sg.tiny_scene(4000, 64, 48, 71, log_scale_mu=-3.3, n_models=3)
    rng = np.random.default_rng(71)
    cams = [sg.look_at(3.0 * sg.random_direction(rng), 64, 48), sg.look_at(3.0 * sg.random_direction(rng), 40, 56)]
    w = sg.Workload("layout", base.models, cams, sg.random_edits(base.models, seed=72),
                    bg=np.array([0.1, 0.2, 0.05], np.float32))
    rast, comp, table = _gpu.setup(w)
    img0 = rast.forward(comp, table).clone()
    dl = torch.randn(img0.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    g0, e0 = rast.backward(comp, table, dl)
    g0 = {k: getattr(g0, k).clone() for k in ATTRS}
    e0 = e0.clone()

    re, order = reorder_spatial(comp)
    o = order.long()
    assert torch.equal(torch.sort(o).values, torch.arange(comp.n, device=o.device))
    mid = re.model_id.long()
    assert bool((mid[1:] >= mid[:-1]).all())
    for k in ATTRS:
        assert torch.equal(getattr(re, k), getattr(comp, k)[o])
    img1 = rast.forward(re, table).clone()
    torch.cuda.synchronize()
    assert torch.equal(img1, img0)
    g1, e1 = rast.backward(re, table, dl)
    for k in ATTRS:
        a, b = getattr(g1, k), g0[k][o]
        assert float((a - b).abs().max()) <= 1e-5 * max(1.0, float(b.abs().max())), k
    assert float((e1 - e0).abs().max()) <= 1e-5 * max(1.0, float(e0.abs().max()))

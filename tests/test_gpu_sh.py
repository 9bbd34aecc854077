"""3DGS colour (SH of the view direction, Sec. 3 / Sec. 4.2) on the GPU against the FP64 oracle:
images, gradients of every attribute and of the SH coefficients, and the edit gradients, for
SH degrees 1 and 3, two views, opacity edits."""
import numpy as np
import pytest
import torch

import oracle
import scenegen as sg
from tests import _gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("deg", [1, 3])
def test_sh_colour_matches_oracle(deg):
    base = sg.tiny_scene(2500, 64, 48, 95, log_scale_mu=-3.3, n_models=2)
    rng = np.random.default_rng(95)
    cams = [sg.look_at(3.0 * sg.random_direction(rng), 64, 48), sg.look_at(3.0 * sg.random_direction(rng), 48, 40)]
    ed = sg.random_edits(base.models, seed=96)
    bg = np.array([0.1, 0.0, 0.2], np.float32)
    w = sg.Workload("sh", base.models, cams, ed, bg=bg)
    M = len(w.models)
    comp_o = oracle.compose(w.models)
    nb = (deg + 1) ** 2
    sh = rng.normal(0, 0.3, (comp_o.n, nb, 3)).astype(np.float32)
    sh[:, 0, :] = rng.uniform(-0.8, 1.6, (comp_o.n, 3))
    comp_o.sh, comp_o.sh_degree = sh.astype(np.float64), deg
    rast, comp, table = _gpu.setup(w)
    comp.sh, comp.sh_degree = torch.as_tensor(sh).cuda().contiguous(), deg
    rast.forward(comp, table)
    dls = [rng.normal(0, 1, (c.H, c.W, 4)) for c in cams]
    dl = torch.as_tensor(np.concatenate([d.reshape(-1, 4) for d in dls]), dtype=torch.float32, device="cuda")
    grad, egrad = rast.backward(comp, table, dl.contiguous())
    torch.cuda.synchronize()
    ref = oracle.render(None, None, cams, bg=bg, comp=comp_o, table=oracle.edit_table(ed))
    for v, c in enumerate(cams):
        unc = _gpu.uncertain_records(ref.projs[v])
        extra = _gpu.uncertain_tile_mask(ref.projs[v], unc, c.W, c.H)
        err, excused, bad = _gpu.compare_image(rast.view_image(v).cpu().numpy(), ref.images[v], ref.margins[v], extra)
        assert bad == 0, (v, err)
    gref = oracle.render_backward(ref, cams, dls, bg=bg)
    for k in ("mean", "log_scale", "quat", "opacity_logit"):
        _gpu.assert_grad(getattr(grad, k).cpu().numpy(), gref.params[k], k)
    for k in ("dcolor", "normal", "kads"):  # not used by the SH colour
        assert float(getattr(grad, k).abs().max()) == 0.0 and np.abs(gref.params[k]).max() == 0.0, k
    _gpu.assert_grad(grad.sh.cpu().numpy(), gref.params["sh"], "sh")
    _gpu.assert_grad(egrad.cpu().numpy()[:len(gref.edit)], gref.edit, "edit table")

"""Precision pattern: Gaussian attributes stored in 16-bit floats (FP16 position offsets from
per-chunk FP32 anchors, BF16 log-scale / colour offset / normal, FP16 quaternion / opacity /
k), all arithmetic in float32.

* The GPU packer (ivrgs_morton_keys + ivrgs_pack_mixed) equals the independent NumPy encoding
  of the storage format bit for bit (order, anchors, every 16-bit value).
* Parity: the same packed arrays rendered on the GPU and by the FP64 oracle on their decoded
  values: images within 2e-4, gradients within 1e-3 relative (kernel error).
* Quantisation error (decoded vs original float32 parameters) is reported separately.
"""
import numpy as np
import pytest
import torch

import oracle
import scenegen as sg
from paper_2504_17954_gb300 import Gaussians, Rasterizer, compose_edit, pack_mixed
from paper_2504_17954_gb300 import _native as N
from tests import _gpu

pytestmark = pytest.mark.gpu


def _composed_arrays(models):
    cat = lambda k: np.concatenate([getattr(m, k) for m in models]).astype(np.float32)
    mid = np.concatenate([np.full(m.n, i, np.int16) for i, m in enumerate(models)])
    return {k: cat(k) for k in sg.ATTRS}, mid


def _upload_packed(p, n_models):
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to("cuda").view(dt)
    return Gaussians(mean=t(p["mean"], torch.float16), log_scale=t(p["log_scale"].view(np.int16), torch.bfloat16),
                     quat=t(p["quat"], torch.float16), opacity_logit=t(p["opacity_logit"], torch.float16),
                     dcolor=t(p["dcolor"].view(np.int16), torch.bfloat16),
                     normal=t(p["normal"].view(np.int16), torch.bfloat16), kads=t(p["kads"], torch.float16),
                     model_id=t(p["model_id"], torch.int16), n_models=n_models, precision=N.IVRGS_MIXED,
                     anchor=t(p["anchor"], torch.float32))


def test_gpu_pack_matches_reference_encoding():
    w = sg.tiny_scene(5000, 32, 32, 41, n_models=3)
    arrs, mid = _composed_arrays(w.models)
    ref, order = sg.pack_mixed_arrays(**arrs, model_id=mid)
    g = Gaussians.from_arrays(arrs, n_models=3)
    g.model_id = torch.as_tensor(mid).cuda()
    packed, gorder = pack_mixed(g)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(gorder.cpu().numpy(), order.astype(np.int32))
    np.testing.assert_array_equal(packed.anchor.cpu().numpy(), ref["anchor"])
    for k in ("mean", "quat", "opacity_logit", "kads"):
        np.testing.assert_array_equal(getattr(packed, k).cpu().view(torch.int16).numpy().reshape(-1),
                                      ref[k].view(np.int16).reshape(-1), err_msg=k)
    for k in ("log_scale", "dcolor", "normal"):
        np.testing.assert_array_equal(getattr(packed, k).cpu().view(torch.int16).numpy().reshape(-1),
                                      ref[k].view(np.int16).reshape(-1), err_msg=k)
    np.testing.assert_array_equal(packed.model_id.cpu().numpy(), ref["model_id"])


@pytest.mark.parametrize("which", ["multi", "cfg1"])
def test_mixed_storage_parity_forward_backward(which):
    if which == "cfg1":
        w = sg.config1()
    else:
        base = sg.tiny_scene(2000, 64, 48, 43, log_scale_mu=-3.3, n_models=3)
        rng = np.random.default_rng(43)
        cams = [sg.look_at(3.0 * sg.random_direction(rng), 64, 48),
                sg.look_at(3.0 * sg.random_direction(rng), 40, 56, headlight=False,
                           light_dir=sg.orbital_light(25.0, 0.4))]
        w = sg.Workload("mixed", base.models, cams, sg.random_edits(base.models, seed=44),
                        bg=np.array([0.1, 0.2, 0.05], np.float32))
    M = len(w.models)
    arrs, mid = _composed_arrays(w.models)
    packed, order = sg.pack_mixed_arrays(**arrs, model_id=mid)
    dec = sg.decode_mixed_arrays(packed)
    g = _upload_packed(packed, M)
    ed = w.edits
    _, table = compose_edit(None, ed.palette, ed.opacity_scale, ed.visible, ed.lam, ed.bias)
    rast = Rasterizer(w.cameras, g.n, M, bg=w.bg)
    rast.forward(g, table)
    rng = np.random.default_rng(45)
    dls = [rng.normal(0, 1, (c.H, c.W, 4)) for c in w.cameras]
    dl = torch.as_tensor(np.concatenate([d.reshape(-1, 4) for d in dls]), dtype=torch.float32, device="cuda")
    grad, egrad = rast.backward(g, table, dl.contiguous())
    torch.cuda.synchronize()
    comp = oracle.Composed(*(np.ascontiguousarray(dec[k], np.float64) for k in oracle.PARAMS),
                           model_id=np.ascontiguousarray(packed["model_id"].astype(np.int32)), n_models=M)
    tab = oracle.edit_table(ed)
    ref = oracle.render(None, None, w.cameras, bg=w.bg, comp=comp, table=tab)
    for v, c in enumerate(w.cameras):
        unc = _gpu.uncertain_records(ref.projs[v])
        extra = _gpu.uncertain_tile_mask(ref.projs[v], unc, c.W, c.H)
        err, excused, bad = _gpu.compare_image(rast.view_image(v).cpu().numpy(), ref.images[v], ref.margins[v], extra)
        assert bad == 0, (v, err)
    gref = oracle.render_backward(ref, w.cameras, dls, bg=w.bg)
    for k in oracle.PARAMS:
        _gpu.assert_grad(getattr(grad, k).cpu().numpy(), gref.params[k], k)
    _gpu.assert_grad(egrad.cpu().numpy()[:len(gref.edit)], gref.edit, "edit table")


def test_quantisation_error_of_mixed_storage_is_small():
    w = sg.config1()
    rast32, comp32, table = _gpu.setup(w)
    img32 = rast32.forward(comp32, table).clone()
    comp32.model_id = comp32.model_id  # composed ids from compose_edit
    packed, _ = pack_mixed(comp32)
    rastm = Rasterizer(w.cameras, packed.n, len(w.models), bg=w.bg)
    imgm = rastm.forward(packed, table)
    torch.cuda.synchronize()
    d = (imgm - img32).abs()
    mse = float((d[:, :3] ** 2).mean())
    psnr = 10 * np.log10(1.0 / max(mse, 1e-20))
    print(f"mixed vs float32 storage: max |d| {float(d.max()):.3e}, PSNR {psnr:.1f} dB")
    assert psnr > 40.0

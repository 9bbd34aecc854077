"""Vector-quantised storage (Sec. 4.4; IVRGS_VQ) on the GPU.

* ivrgs_vq_build (k-means on the device) against the FP64 oracle's k-means: codebooks within
  1e-4 of each attribute's value range; indices equal except where a value sits within rounding
  of a midpoint, and there the GPU's centroid is as near as the oracle's.
* Rendering from VQ storage (indices and codebooks built by the oracle): images, gradients and
  auxiliary maps against the FP64 oracle on the decoded values (kernel error).
* Quantisation error of k = 256 codebooks on the 10k-Gaussian scene, reported with a floor.
"""
import numpy as np
import pytest
import torch

import oracle
import scenegen as sg
from oracle import vq as ovq
from paper_2504_17954_gb300 import Gaussians, Rasterizer, compose_edit, vq_compress
from paper_2504_17954_gb300 import _native as N
from tests import _gpu
from tests.test_gpu_mixed import _composed_arrays

pytestmark = pytest.mark.gpu


def _fp32_composed(w):
    arrs, mid = _composed_arrays(w.models)
    g = Gaussians.from_arrays(arrs, n_models=len(w.models))
    g.model_id = torch.as_tensor(mid).cuda()
    return g, arrs, mid


def test_vq_build_matches_oracle():
    w = sg.tiny_scene(6000, 32, 32, 91, n_models=3)
    g, arrs, mid = _fp32_composed(w)
    K, iters = 64, 6
    q = vq_compress(g, k=K, iters=iters)
    torch.cuda.synchronize()
    cb_o, idx_o = ovq.build({k: v.astype(np.float64) for k, v in arrs.items()}, mid, len(w.models), K, iters)
    cb_g = q.codebook.cpu().numpy().astype(np.float64)
    for m in range(len(w.models)):
        for a in range(N.IVRGS_VQ_ATTRS):
            rng_ = max(float(cb_o[m, a].max() - cb_o[m, a].min()), 1e-6)
            assert np.abs(cb_g[m, a] - cb_o[m, a]).max() <= 1e-4 * rng_, (m, a)
    names = ("log_scale", "quat", "opacity_logit", "dcolor", "kads")
    agree, total = 0, 0
    for nm in names:
        gi = getattr(q, nm).cpu().numpy().reshape(idx_o[nm].shape)
        oi = idx_o[nm]
        agree += int((gi == oi).sum())
        total += gi.size
        # where they differ, the GPU's centroid is (to rounding) as near as the oracle's
        bad = np.nonzero(gi != oi)
        for pos in zip(*bad):
            i = pos[0]
            comp = pos[1] if len(pos) > 1 else 0
            a = {"log_scale": 0, "quat": 1, "opacity_logit": 2, "dcolor": 3}.get(nm, 4 + comp)
            v = float(arrs[nm][pos]) if arrs[nm].ndim > 1 else float(arrs[nm][i])
            c = cb_g[mid[i], a]
            assert abs(abs(v - c[gi[pos]]) - abs(v - c[oi[pos]])) <= 1e-5 * max(1.0, abs(v)), (nm, pos)
    assert agree >= 0.995 * total, (agree, total)


def _upload_vq(w, k=64, iters=6):
    arrs, mid = _composed_arrays(w.models)
    M = len(w.models)
    cb, idx = ovq.build({kk: v.astype(np.float64) for kk, v in arrs.items()}, mid, M, k, iters)
    cb32 = cb.astype(np.float32)
    dec = ovq.decode(cb32.astype(np.float64), idx, mid)
    t = lambda a, dt=None: torch.as_tensor(np.ascontiguousarray(a)).cuda() if dt is None else \
        torch.as_tensor(np.ascontiguousarray(a, dt)).cuda()
    g = Gaussians(mean=t(arrs["mean"], np.float32), log_scale=t(idx["log_scale"]), quat=t(idx["quat"]),
                  opacity_logit=t(idx["opacity_logit"]), dcolor=t(idx["dcolor"]), normal=t(arrs["normal"], np.float32),
                  kads=t(idx["kads"]), model_id=t(mid), n_models=M, precision=N.IVRGS_VQ, codebook=t(cb32), vq_k=k)
    dec["mean"] = arrs["mean"].astype(np.float64)
    dec["normal"] = arrs["normal"].astype(np.float64)
    return g, dec, mid


@pytest.mark.parametrize("which", ["cfg1", "multi"])
def test_vq_storage_parity(which):
    if which == "cfg1":
        w = sg.config1()
    else:
        base = sg.tiny_scene(2500, 64, 48, 92, log_scale_mu=-3.3, n_models=3)
        rng = np.random.default_rng(92)
        cams = [sg.look_at(3.0 * sg.random_direction(rng), 64, 48),
                sg.look_at(3.0 * sg.random_direction(rng), 40, 56, headlight=False,
                           light_dir=sg.orbital_light(25.0, 0.4))]
        w = sg.Workload("vq", base.models, cams, sg.random_edits(base.models, seed=93),
                        bg=np.array([0.1, 0.2, 0.05], np.float32))
    M = len(w.models)
    g, dec, mid = _upload_vq(w)
    ed = w.edits
    _, table = compose_edit(None, ed.palette, ed.opacity_scale, ed.visible, ed.lam, ed.bias)
    rast = Rasterizer(w.cameras, g.n, M, bg=w.bg)
    rast.forward(g, table)
    rng = np.random.default_rng(94)
    dls = [rng.normal(0, 1, (c.H, c.W, 4)) for c in w.cameras]
    dl = torch.as_tensor(np.concatenate([d.reshape(-1, 4) for d in dls]), dtype=torch.float32, device="cuda")
    grad, egrad = rast.backward(g, table, dl.contiguous())
    aux = rast.render_aux(g, table).clone()
    torch.cuda.synchronize()
    comp = oracle.Composed(*(np.ascontiguousarray(dec[k], np.float64) for k in oracle.PARAMS),
                           model_id=np.ascontiguousarray(mid.astype(np.int32)), n_models=M)
    tab = oracle.edit_table(ed)
    ref = oracle.render(None, None, w.cameras, bg=w.bg, comp=comp, table=tab)
    maps = oracle.render_aux(ref, w.cameras)
    for v, c in enumerate(w.cameras):
        unc = _gpu.uncertain_records(ref.projs[v])
        extra = _gpu.uncertain_tile_mask(ref.projs[v], unc, c.W, c.H)
        err, excused, bad = _gpu.compare_image(rast.view_image(v).cpu().numpy(), ref.images[v], ref.margins[v], extra)
        assert bad == 0, (v, err)
        off = rast.cam_arr[v].pix_offset
        ga = aux[off:off + c.W * c.H].cpu().numpy().reshape(c.H, c.W, 12)
        ex = _gpu.near_tie(ref.margins[v]) | extra
        for k in range(12):
            s = max(1.0, float(np.abs(maps[v][..., k]).max()))
            e = np.abs(ga[..., k] - maps[v][..., k]) / s
            assert not ((e > 2e-4) & ~ex).any(), (v, k)
    gref = oracle.render_backward(ref, w.cameras, dls, bg=w.bg)
    for k in oracle.PARAMS:
        _gpu.assert_grad(getattr(grad, k).cpu().numpy(), gref.params[k], k)
    _gpu.assert_grad(egrad.cpu().numpy()[:len(gref.edit)], gref.edit, "edit table")


def test_vq_quantisation_error():
    w = sg.config1()
    rast32, comp32, table = _gpu.setup(w)
    img32 = rast32.forward(comp32, table).clone()
    q = vq_compress(comp32, k=256, iters=16)
    rq = Rasterizer(w.cameras, q.n, len(w.models), bg=w.bg)
    imgq = rq.forward(q, table)
    torch.cuda.synchronize()
    mse = float(((imgq - img32)[:, :3] ** 2).mean())
    psnr = 10 * np.log10(1.0 / max(mse, 1e-20))
    bytes_fp32 = 86
    bytes_vq = 12 + 12 + 2 + 15
    print(f"VQ k=256: PSNR {psnr:.1f} dB vs float32 storage, {bytes_vq} vs {bytes_fp32} bytes per Gaussian")
    assert psnr > 35.0

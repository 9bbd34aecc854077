"""Inverse volume exploration on the GPU (Sec. 4.6) against the FP64 oracle (oracle/inverse.py).

* ivrgs_image_loss: loss, L1, SSIM and dloss/dRGB on two packed views of ragged sizes (the
  plain L1 loss, lambda_ssim = 0, skips SSIM).
* ivrgs_edit_adam: two steps on a random table and gradient (all parameter groups, light on).
* One whole iteration (render, loss, backward, Adam) from the same edits and the same
  oracle-rendered reference: loss, edit gradients (incl. the light direction) and the update.
* Fitting: from perturbed edits, 300 graph-replayed iterations bring the rendering close to an
  oracle-rendered reference made with other colours, opacities, light magnitude and direction.
"""
import numpy as np
import pytest
import torch

import oracle
import scenegen as sg
from oracle import inverse as oinv
from paper_2504_17954_gb300 import _native as N
from paper_2504_17954_gb300.inverse import LEARN_ALL, InverseExplorer
from paper_2504_17954_gb300.rasterizer import _stream, _vp, camera_structs
from tests import _gpu

pytestmark = pytest.mark.gpu


def test_image_loss_matches_oracle():
    cams = [sg.look_at([3, 0, 0], 37, 29), sg.look_at([0, 3, 0], 64, 48)]
    arr, n_pix = camera_structs(cams)
    rng = np.random.default_rng(61)
    x = rng.random((n_pix, 4)).astype(np.float32)
    y = rng.random((n_pix, 4)).astype(np.float32)
    xs, ys = [], []
    for v, c in enumerate(cams):
        o = arr[v].pix_offset
        xs.append(x[o:o + c.W * c.H].reshape(c.H, c.W, 4).astype(np.float64))
        ys.append(y[o:o + c.W * c.H].reshape(c.H, c.W, 4).astype(np.float64))
    for lam in (0.2, 0.0, 1.0):
        loss, l1, ssim, grads = oinv.image_loss(xs, ys, lam)
        dx, dy = torch.as_tensor(x, device="cuda"), torch.as_tensor(y, device="cuda")
        wsb = N.ivrgs_image_loss_workspace(arr, len(cams))
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        out = torch.zeros(3, dtype=torch.float32, device="cuda")
        dL = torch.full((n_pix, 4), 7.0, dtype=torch.float32, device="cuda")
        N.ivrgs_image_loss(_vp(dx), _vp(dy), arr, len(cams), lam, _vp(ws), wsb, _vp(out), _vp(dL), _stream())
        torch.cuda.synchronize()
        o = out.cpu().numpy().astype(np.float64)
        assert abs(o[0] - loss) <= 1e-6 * max(1.0, abs(loss)), (lam, o, loss)
        assert abs(o[1] - l1) <= 1e-6, (o, l1)
        if lam == 0.0:  # the plain L1 loss: SSIM not evaluated
            assert o[2] == 0.0
        else:
            assert abs(o[2] - ssim) <= 1e-6, (o, ssim)
        g = dL.cpu().numpy()
        for v, c in enumerate(cams):
            off = arr[v].pix_offset
            gv = g[off:off + c.W * c.H].reshape(c.H, c.W, 4)
            assert np.all(gv[..., 3] == 0.0)
            assert _gpu.rel_l2(gv[..., :3].astype(np.float64), grads[v]) < 1e-4, (lam, v)


def test_adam_matches_oracle():
    M = 3
    rng = np.random.default_rng(62)
    table = np.zeros(8 * M + 12)
    for m in range(M):
        table[8 * m:8 * m + 5] = [*rng.random(3), rng.uniform(0.5, 1.5), 1.0]
    table[8 * M:8 * M + 8] = [*rng.uniform(0.8, 1.2, 4), *rng.normal(0, 0.05, 4)]
    table[8 * M + 8:8 * M + 12] = [*oinv.light_dir(0.9, 2.1), 1.0]
    table = table.astype(np.float32).astype(np.float64)
    dt = torch.as_tensor(table.astype(np.float32), device="cuda")
    st_g = torch.empty(N.lib().ivrgs_edit_adam_state_floats(M), dtype=torch.float32, device="cuda")
    N.ivrgs_edit_adam_init(_vp(dt), M, _vp(st_g), _stream())
    st_o = oinv.AdamState(table, M)
    tab_o = table.copy()
    for k in range(3):
        eg = rng.normal(0, 1, 8 * M + 12 + 4).astype(np.float32)
        deg = torch.as_tensor(eg, device="cuda")
        N.ivrgs_edit_adam(_vp(dt), _vp(deg), M, _vp(st_g), LEARN_ALL, 0.01, 0.9, 0.999, 1e-8, _stream())
        tab_o = oinv.adam_step(tab_o, eg[:8 * M + 12].astype(np.float64), M, st_o, LEARN_ALL, 0.01)
    torch.cuda.synchronize()
    np.testing.assert_allclose(dt.cpu().numpy(), tab_o, rtol=0, atol=2e-6)
    s = st_g.cpu().numpy()
    P = 4 * M + 10
    np.testing.assert_allclose(s[2 * P:2 * P + 2], st_o.angles, rtol=0, atol=2e-6)
    assert s[-1] == 3.0


def _inverse_scene():
    w = sg.tiny_scene(2500, 64, 56, 63, log_scale_mu=-3.2, headlight=False, n_models=3)
    cam = w.cameras[0]
    true = sg.random_edits(w.models, seed=64)
    true.lam = np.array([1.2, 0.8, 1.1, 0.9], np.float32)
    true.bias = np.array([0.05, -0.02, 0.03, 2.0], np.float32)
    true.light_dir = oinv.light_dir(1.0, 0.8)
    start = sg.identity_edits(w.models)
    start.light_dir = oinv.light_dir(1.3, 0.4)
    bg = np.array([0.05, 0.05, 0.1], np.float32)
    return sg.Workload("inverse", w.models, [cam], start, bg=bg), true


def _upload_reference(w, true):
    ref = oracle.render(w.models, true, w.cameras, bg=w.bg)
    return ref, torch.as_tensor(ref.images[0].reshape(-1, 4).astype(np.float32), device="cuda").contiguous()


def test_one_iteration_matches_oracle():
    w, true = _inverse_scene()
    _, target = _upload_reference(w, true)
    rast, comp, table = _gpu.setup(w)
    table0 = table.cpu().numpy().astype(np.float64)
    ex = InverseExplorer(rast, comp, table, target, learn=LEARN_ALL, lr=0.01)
    ex.step()
    torch.cuda.synchronize()
    # oracle: the same iteration from the same table
    M = len(w.models)
    r = oracle.render(w.models, w.edits, w.cameras, bg=w.bg, table=table0)
    tgt = target.cpu().numpy().astype(np.float64).reshape(w.cameras[0].H, w.cameras[0].W, 4)
    loss, l1, ssim, grads = oinv.image_loss([r.images[0]], [tgt], 0.2)
    assert abs(float(ex.loss[0]) - loss) <= 2e-4 * loss, (float(ex.loss[0]), loss)
    dl = np.concatenate([grads[0], np.zeros(grads[0].shape[:2] + (1,))], -1)
    gr = oracle.render_backward(r, w.cameras, [dl], bg=w.bg)
    eg = rast.edit_grad.cpu().numpy().astype(np.float64)
    for m in range(M):
        assert _gpu.rel_l2(eg[8 * m:8 * m + 4], gr.edit[8 * m:8 * m + 4]) < 2e-3, m
    assert _gpu.rel_l2(eg[8 * M:8 * M + 8], gr.edit[8 * M:8 * M + 8]) < 2e-3
    assert _gpu.rel_l2(eg[8 * M + 8:8 * M + 11], gr.edit[8 * M + 8:8 * M + 11]) < 2e-3
    # the update: the oracle's Adam on the GPU's gradients gives the GPU's table
    st = oinv.AdamState(table0, M)
    tab1 = oinv.adam_step(table0, eg[:8 * M + 12], M, st, LEARN_ALL, 0.01)
    np.testing.assert_allclose(table.cpu().numpy(), tab1, rtol=0, atol=2e-6)
    assert ex.step_count() == 1


def test_fitting_recovers_the_reference():
    w, true = _inverse_scene()
    ref, target = _upload_reference(w, true)
    rast, comp, table = _gpu.setup(w)
    ex = InverseExplorer(rast, comp, table, target, learn=LEARN_ALL, lr=0.01)
    hist = ex.run(300, graph=True, record_every=50)
    torch.cuda.synchronize()
    print("loss every 50 iterations:", [f"{h:.4f}" for h in hist])
    assert ex.step_count() == 300
    # Adam at a constant learning rate wanders near the optimum once it is reached, so the fit is
    # judged by the lowest loss of the run (sampled every 50 iterations) and the final rendering
    assert min(hist[1:]) < 0.25 * hist[0], hist
    rast.forward(comp, table)
    torch.cuda.synchronize()
    img = rast.view_image(0).cpu().numpy()[..., :3].astype(np.float64)
    mse = float(((img - ref.images[0][..., :3]) ** 2).mean())
    psnr = 10 * np.log10(1.0 / mse)
    print(f"PSNR of the fitted rendering vs the reference: {psnr:.1f} dB")
    assert psnr > 30.0
    # the light direction stays a unit vector written from its angles
    M = len(w.models)
    L = table.cpu().numpy()[8 * M + 8:8 * M + 11]
    assert abs(np.linalg.norm(L) - 1.0) < 1e-5
    th, ph = ex.light_angles()
    np.testing.assert_allclose(L, oinv.light_dir(th, ph), atol=1e-5)

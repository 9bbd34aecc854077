"""Views rendered in waves (each binning call stays under the per-call pair limit) with the
backward summed across waves by ivrgs_render_backward_accumulate.

* Waves vs one call: the same images bit for bit and the same gradients (1e-5 relative); the
  shape (tile height and waves) picked by the autotuner renders the images of one call.
* The 3M-Gaussian / 8-model / 64-view workload (sides 512..2048) in 16-bit storage, the batched
  mixed-precision form: sampled pixels of a 4-view subset and the gradients of a loss on them
  against the FP64 oracle on the decoded values; the same views rendered from float32 storage
  give the quantisation error (PSNR), reported.
"""
import numpy as np
import pytest
import torch

import oracle
import scenegen as sg
from paper_2504_17954_gb300 import Gaussians, compose_edit
from paper_2504_17954_gb300.rasterizer import Rasterizer, WaveRasterizer
from tests import _gpu

pytestmark = pytest.mark.gpu


def test_waves_equal_one_call():
    base = sg.tiny_scene(4000, 64, 48, 51, log_scale_mu=-3.3, n_models=2)
    rng = np.random.default_rng(51)
    cams = [sg.look_at(3.0 * sg.random_direction(rng), 40 + 8 * i, 48, headlight=i % 2 == 0,
                       light_dir=sg.orbital_light(10.0 * i, 0.2 * i)) for i in range(6)]
    w = sg.Workload("waves", base.models, cams, sg.random_edits(base.models, seed=52))
    one, comp, table = _gpu.setup(w)
    one.forward(comp, table)
    waves = WaveRasterizer(cams, comp.n, 2, max_views=2)
    assert len(waves.waves) == 3
    waves.forward(comp, table)
    dls = [torch.as_tensor(rng.normal(0, 1, (c.H * c.W, 4)), dtype=torch.float32, device="cuda") for c in cams]
    g1, e1 = one.backward(comp, table, torch.cat(dls).contiguous())
    g1 = {k: getattr(g1, k).clone() for k in ("mean", "log_scale", "quat", "opacity_logit", "dcolor", "normal",
                                              "kads")}
    e1 = e1.clone()
    per_wave = [torch.cat([dls[v] for v in wv]).contiguous() for wv in waves.waves]
    g2, e2, light = waves.backward(comp, table, per_wave)
    torch.cuda.synchronize()
    for v in range(len(cams)):
        assert torch.equal(one.view_image(v), waves.view_image(v))
    for k, ref in g1.items():
        assert float((getattr(g2, k) - ref).norm() / ref.norm()) < 1e-5, k
    ne = table.numel()
    assert float((e2 - e1[:ne]).norm() / e1[:ne].norm()) < 1e-5
    ref_light = e1[ne:].view(len(cams), 4)[:, :3]
    assert float((light - ref_light).norm() / ref_light.norm()) < 1e-5


def test_tuned_wave_shape_renders_the_same_views():
    """autotune.tune_waves on a 6-view scene with small pixel budgets and both tile heights: it
    times each distinct shape (captured forward+backward), and the picked shape renders every view
    bit for bit as one call with the same tile height does."""
    from paper_2504_17954_gb300 import autotune
    base = sg.tiny_scene(4000, 64, 48, 53, log_scale_mu=-3.3, n_models=2)
    rng = np.random.default_rng(53)
    cams = [sg.look_at(3.0 * sg.random_direction(rng), 40 + 8 * i, 48) for i in range(6)]
    w = sg.Workload("tune", base.models, cams, sg.random_edits(base.models, seed=54))
    timed = []

    def measure(mv, pb, th):
        wv = WaveRasterizer(cams, 4000, 2, max_views=mv, pixel_budget=pb, tile_h=th)
        _, comp, table = _gpu.setup(w, tile_h=th)
        wv.size_buffers(comp, table)
        dls = [torch.zeros((r.n_pix, 4), device="cuda") for r in wv.rasts]
        graph = wv.capture(comp, table, dls)
        graph.replay()
        torch.cuda.synchronize()
        ms = autotune.time_ms(graph.replay, reps=3)
        timed.append((th, len(wv.waves)))
        return ms
    budgets = (4000, 8000, 16000)
    shape = autotune.tune_waves(measure, cams, 4000, "test", budgets=budgets, max_views=(2, 32),
                                tile_heights=(16, 8), use_cache=False)
    assert len(timed) == len({(c["tile_h"], tuple(c["waves"])) for c in shape["candidates"]}) >= 6
    assert shape["ms"] == min(c["ms"] for c in shape["candidates"])
    th = shape["tile_h"]
    one, comp, table = _gpu.setup(w, tile_h=th)
    one.forward(comp, table)
    waves = WaveRasterizer(cams, comp.n, 2, max_views=shape["max_views"], pixel_budget=shape["pixel_budget"],
                           tile_h=th)
    assert [len(x) for x in waves.waves] == shape["waves"]
    waves.forward(comp, table)
    torch.cuda.synchronize()
    for v in range(len(cams)):
        assert torch.equal(one.view_image(v), waves.view_image(v))


def _upload(p, M):
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to("cuda").view(dt)
    return Gaussians(mean=t(p["mean"], torch.float16), log_scale=t(p["log_scale"].view(np.int16), torch.bfloat16),
                     quat=t(p["quat"], torch.float16), opacity_logit=t(p["opacity_logit"], torch.float16),
                     dcolor=t(p["dcolor"].view(np.int16), torch.bfloat16),
                     normal=t(p["normal"].view(np.int16), torch.bfloat16), kads=t(p["kads"], torch.float16),
                     model_id=t(p["model_id"], torch.int16), n_models=M, precision=1,
                     anchor=t(p["anchor"], torch.float32))


def test_3m_64_views_mixed_storage_in_waves():
    w = sg.config5()
    M = len(w.models)
    cat = lambda k: np.concatenate([getattr(m, k) for m in w.models]).astype(np.float32)
    arrs = {k: cat(k) for k in sg.ATTRS}
    mid = np.concatenate([np.full(m.n, i, np.int16) for i, m in enumerate(w.models)])
    packed, _ = sg.pack_mixed_arrays(**arrs, model_id=mid)
    g = _upload(packed, M)
    ed = w.edits
    _, table = compose_edit(None, ed.palette, ed.opacity_scale, ed.visible, ed.lam, ed.bias)
    waves = WaveRasterizer(w.cameras, g.n, M, bg=w.bg, pixel_budget=12 << 20)
    waves.forward(g, table)
    torch.cuda.synchronize()
    assert len(waves.waves) >= 4
    dec = sg.decode_mixed_arrays(packed)
    comp = oracle.Composed(*(np.ascontiguousarray(dec[k], np.float64) for k in oracle.PARAMS),
                           model_id=np.ascontiguousarray(packed["model_id"].astype(np.int32)), n_models=M)
    tab = oracle.edit_table(ed)
    subset = [0, 21, 42, 63]
    rng = np.random.default_rng(53)
    pix_v, dl_v, projs, excused = {}, {}, {}, 0
    for v in subset:
        c = w.cameras[v]
        p = oracle.project(comp, tab, c)
        pix = np.c_[rng.integers(0, c.W, 96), rng.integers(0, c.H, 96)]
        rgba, T, last, mg = oracle.render_pixels(p, c, pix, bg=w.bg)
        gimg = waves.view_image(v).cpu().numpy()[pix[:, 1], pix[:, 0]]
        unc = _gpu.uncertain_records(p)
        tile_unc = _gpu.uncertain_tile_mask(p, unc, c.W, c.H)[pix[:, 1], pix[:, 0]]
        err, exc, bad = _gpu.compare_image(gimg, rgba, mg, tile_unc)
        assert bad == 0, (v, err)
        excused += exc
        safe = ~(_gpu.near_tie(mg) | tile_unc)
        pick = pix[safe][:32]
        _, uniq = np.unique(pick[:, 1] * c.W + pick[:, 0], return_index=True)
        pix_v[v], projs[v] = pick[np.sort(uniq)], p
        dl_v[v] = rng.normal(0, 1, (len(pix_v[v]), 4))
    assert excused <= 2
    # gradients of a loss on the sampled pixels, summed over the waves
    per_wave = []
    for r, wv in zip(waves.rasts, waves.waves):
        d = np.zeros((r.n_pix, 4), np.float32)
        for j, v in enumerate(wv):
            if v in pix_v:
                off, c = r.cam_arr[j].pix_offset, w.cameras[v]
                d[off + pix_v[v][:, 1] * c.W + pix_v[v][:, 0]] = dl_v[v]
        per_wave.append(torch.as_tensor(d, device="cuda"))
    grad, eg, light = waves.backward(g, table, per_wave)
    torch.cuda.synchronize()
    ref = oracle.pixels_backward(comp, tab, [w.cameras[v] for v in subset], [projs[v] for v in subset],
                                 [pix_v[v] for v in subset], [dl_v[v] for v in subset], bg=w.bg)
    for k in oracle.PARAMS:
        _gpu.assert_grad(getattr(grad, k).cpu().numpy(), ref.params[k], k)
    _gpu.assert_grad(eg.cpu().numpy(), ref.edit, "edit table")
    # quantisation error of the storage: the same views from float32 storage (original order)
    comp32, _ = compose_edit([Gaussians.from_arrays({k: getattr(m, k) for k in sg.ATTRS}) for m in w.models],
                             ed.palette, ed.opacity_scale, ed.visible, ed.lam, ed.bias)
    r32 = Rasterizer([w.cameras[v] for v in subset], comp32.n, M, bg=w.bg)
    r32.forward(comp32, table)
    torch.cuda.synchronize()
    for j, v in enumerate(subset):
        a, b = waves.view_image(v)[..., :3], r32.view_image(j)[..., :3]
        mse = float(((a - b) ** 2).mean())
        print(f"view {v}: max |mixed - fp32 storage| {float((a - b).abs().max()):.2e}, "
              f"PSNR {10 * np.log10(1 / max(mse, 1e-20)):.1f} dB")
        assert 10 * np.log10(1 / max(mse, 1e-20)) > 40.0

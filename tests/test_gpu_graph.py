"""CUDA-graph capture of a whole step (batching pattern): projection, CAPACITY-mode binning,
compositing and backward recorded once and replayed. Replays after editing the edit table
(palette, opacity scale, a hidden model) must equal eager calls with the same edits: the
forward bit for bit (no atomics), the gradients within 1e-5 relative (atomic order)."""
import numpy as np
import pytest
import torch

import scenegen as sg
from paper_2504_17954_gb300 import compose_edit
from paper_2504_17954_gb300 import autotune
from tests import _gpu

pytestmark = pytest.mark.gpu


def test_graph_replay_matches_eager_across_edits():
    w = sg.tiny_scene(3000, 96, 80, 31, log_scale_mu=-3.2, n_models=3)
    cams = [w.cameras[0], sg.look_at([0.5, 2.5, 1.0], 64, 72, headlight=False,
                                     light_dir=sg.orbital_light(30.0, 1.0))]
    w = sg.Workload("graph", w.models, cams, w.edits)
    rast, comp, table = _gpu.setup(w)
    rast.forward(comp, table, mode="exact")
    rast._ensure_capacity(int(rast.n_pairs * 2) + 4096)
    dl = torch.as_tensor(np.random.default_rng(2).normal(0, 1, (rast.n_pix, 4)), dtype=torch.float32,
                         device="cuda").contiguous()
    graph = rast.capture(comp, table, dl)
    edits = [w.edits, sg.random_edits(w.models, seed=5), sg.random_edits(w.models, seed=6, hide=1)]
    for ed in edits:
        compose_edit(None, ed.palette, ed.opacity_scale, ed.visible, ed.lam, ed.bias, edit_table=table)
        graph.replay()
        torch.cuda.synchronize()
        assert int(rast.d_n_pairs.item()) <= rast.capacity
        g_img = rast.rgba.clone()
        g_grad = {k: getattr(rast.graph_grad, k).clone() for k in ("mean", "log_scale", "opacity_logit", "dcolor")}
        rast.forward(comp, table, mode="exact")
        grad, _ = rast.backward(comp, table, dl)
        torch.cuda.synchronize()
        assert torch.equal(g_img, rast.rgba)
        for k, v in g_grad.items():
            ref = getattr(grad, k)
            assert float((v - ref).norm() / ref.norm()) < 1e-5, k


def test_autotuner_picks_a_valid_choice(tmp_path, monkeypatch):
    monkeypatch.setenv("IVRGS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    w = sg.config1()
    rast, comp, table = _gpu.setup(w)
    rast.forward(comp, table)
    before = autotune.current()
    try:
        choice = autotune.tune(lambda: rast.forward(comp, table, mode="capacity"), "cfg1-test", reps=2,
                               space={"render_pixels_per_thread": (1, 2)})
        assert choice["render_pixels_per_thread"] in (1, 2)
        assert autotune.current()["render_pixels_per_thread"] == choice["render_pixels_per_thread"]
        again = autotune.tune(lambda: None, "cfg1-test")  # served from the cache
        assert again == choice
    finally:
        autotune.apply(before)


def test_graph_with_image_loss_matches_eager():
    """A captured step with the L1 image loss between compositing and backward (the loss of the
    500k-Gaussian single-view benchmark leg) equals the eager forward, loss and backward."""
    from paper_2504_17954_gb300 import _native as N
    from paper_2504_17954_gb300.rasterizer import _stream, _vp
    w = sg.tiny_scene(3000, 96, 80, 33, log_scale_mu=-3.2, n_models=2)
    rast, comp, table = _gpu.setup(w)
    rast.forward(comp, table, mode="exact")
    rast._ensure_capacity(int(rast.n_pairs * 2) + 4096)
    target = torch.rand((rast.n_pix, 4), generator=torch.Generator("cuda").manual_seed(3), device="cuda")
    wsb = N.ivrgs_image_loss_workspace(rast.cam_arr, rast.V)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    out = torch.zeros(3, dtype=torch.float32, device="cuda")
    dl = torch.zeros((rast.n_pix, 4), dtype=torch.float32, device="cuda")

    def l1():
        N.ivrgs_image_loss(_vp(rast.rgba), _vp(target), rast.cam_arr, rast.V, 0.0, _vp(ws), wsb, _vp(out), _vp(dl),
                           _stream())
    graph = rast.capture(comp, table, dl, loss=l1)
    graph.replay()
    torch.cuda.synchronize()
    g_img, g_loss, g_dl = rast.rgba.clone(), out.clone(), dl.clone()
    g_grad = {k: getattr(rast.graph_grad, k).clone() for k in ("mean", "log_scale", "opacity_logit", "dcolor")}
    dl.zero_()
    rast.forward(comp, table, mode="exact")
    l1()
    grad, _ = rast.backward(comp, table, dl)
    torch.cuda.synchronize()
    assert torch.equal(g_img, rast.rgba) and torch.equal(g_dl, dl) and torch.equal(g_loss, out)
    assert float(out[0]) > 0 and float(out[2]) == 0.0
    for k, v in g_grad.items():
        ref = getattr(grad, k)
        assert float((v - ref).norm() / ref.norm()) < 1e-5, k


def test_wave_graph_matches_eager_waves():
    """All waves' forward and backward captured as one graph equal the eager wave calls."""
    from paper_2504_17954_gb300.rasterizer import WaveRasterizer
    base = sg.tiny_scene(4000, 64, 48, 51, log_scale_mu=-3.3, n_models=2)
    rng = np.random.default_rng(54)
    cams = [sg.look_at(3.0 * sg.random_direction(rng), 40 + 8 * i, 48, headlight=i % 2 == 0,
                       light_dir=sg.orbital_light(10.0 * i, 0.2 * i)) for i in range(5)]
    w = sg.Workload("waves", base.models, cams, sg.random_edits(base.models, seed=55))
    _, comp, table = _gpu.setup(w)
    waves = WaveRasterizer(cams, comp.n, 2, max_views=2, bg=(0.1, 0.2, 0.3))
    assert len(waves.waves) == 3
    waves.size_buffers(comp, table)
    dls = [torch.as_tensor(rng.normal(0, 1, (r.n_pix, 4)), dtype=torch.float32, device="cuda").contiguous()
           for r in waves.rasts]
    graph = waves.capture(comp, table, dls)
    graph.replay()
    torch.cuda.synchronize()
    assert not waves.overflowed()
    imgs = [waves.view_image(v).clone() for v in range(len(cams))]
    g_grad = {k: getattr(waves.graph_grad, k).clone() for k in ("mean", "log_scale", "quat", "opacity_logit")}
    g_edit, g_light = waves.edit_grad[:table.numel()].clone(), waves.light_grad.clone()
    waves.forward(comp, table)
    grad, eg, light = waves.backward(comp, table, dls)
    torch.cuda.synchronize()
    for v in range(len(cams)):
        assert torch.equal(imgs[v], waves.view_image(v)), v
    for k, val in g_grad.items():
        ref = getattr(grad, k)
        assert float((val - ref).norm() / ref.norm()) < 1e-5, k
    assert float((g_edit - eg).norm() / eg.norm()) < 1e-5
    assert float((g_light - light).norm() / light.norm()) < 1e-5

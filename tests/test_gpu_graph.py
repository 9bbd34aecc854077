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

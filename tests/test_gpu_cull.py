"""Tile culling by the opacity cut-off ellipse (ivrgs_bin with IVRGS_BIN_CULL).

Every (tile, Gaussian) pair that culling removes must be one that the compositing skips at
every pixel of that tile, so:

* the culled lists are the rectangle lists (themselves checked bit for bit against the oracle
  in test_gpu_parity.py) with pairs removed and the order kept;
* each removed pair is skipped by the FP64 oracle at all pixel centres of its tile:
  min(0.99, o' exp(-q/2)) < 1/255 with the oracle's own conic and opacity;
* images, final transmittances and last contributors are bit-identical with and without
  culling, and the images are within 2e-4 of the FP64 oracle; the gradients differ only by the
  order of their float32 atomic sums: with and without culling they meet the gradient bar
  against the FP64 oracle (1e-3 relative L2 and 1e-3 of the largest entry element by element),
  the thin-Gaussian scene included, and lie within 1e-4 of each other except in that scene
  (where order noise of its sums shows more).

Scenes: the 10k-Gaussian 128^2 case, a three-view scene with colour/opacity/light edits and an
orbital light, a scene whose opacity edits put many o' around 1/255, and a scene with strongly
elongated Gaussians on both sides of the conditioning limit beyond which a Gaussian keeps its
whole rectangle.
"""
import numpy as np
import pytest
import torch

import oracle
import scenegen as sg
from tests import _gpu
from tests.test_gpu_parity import _multi_view_scene

pytestmark = pytest.mark.gpu

ALPHA_MIN = 1.0 / 255.0


def _scene(which):
    if which == "cfg1":
        return sg.config1()
    if which == "multi":
        return _multi_view_scene(seed=31)
    w = sg.tiny_scene(3000, 96, 80, 33, log_scale_mu=-3.0, n_models=3)
    if which == "low_opacity":
        # o' = s_m sigmoid(logit) spread across 1/255 for two of the three models
        w.edits.opacity_scale = np.array([0.004, 0.012, 1.0], np.float32)
        return w
    # elongated: one long axis (world sigma 0.14 .. 1.35) and two tiny ones for half the Gaussians
    r = np.random.default_rng(34)
    for m in w.models:
        sel = r.random(m.n) < 0.5
        m.log_scale[sel, 0] = r.uniform(-2.0, 0.3, sel.sum()).astype(np.float32)
        m.log_scale[sel, 1:] = np.float32(-7.0)
    return w


def _run(w, cull, dl):
    rast, comp, table = _gpu.setup(w, cull=cull)
    rast.forward(comp, table)
    grad, eg = rast.backward(comp, table, dl)
    torch.cuda.synchronize()
    g = {k: getattr(grad, k).clone() for k in oracle.PARAMS}
    return rast, g, eg.clone()


def _tile_lists(rast):
    r = rast.ranges.cpu().numpy().view(np.uint32).astype(np.int64)
    vals = rast.values.cpu().numpy().view(np.uint32)
    return [vals[a:b] for a, b in r]


def _max_alpha_over_tile(p, cam, g, tx, ty):
    """FP64: largest alpha of Gaussians g over the pixel centres of tiles (tx, ty) of one view."""
    out = np.zeros(len(g))
    for s in range(0, len(g), 4096):
        gg, xx, yy = g[s:s + 4096], tx[s:s + 4096], ty[s:s + 4096]
        ii = np.arange(16)
        px = 16 * xx[:, None, None] + ii[None, None, :] + 0.5   # [k, 1, 16]
        py = 16 * yy[:, None, None] + ii[None, :, None] + 0.5   # [k, 16, 1]
        inside = (px < cam.W) & (py < cam.H)
        dx = p.uv[gg, 0][:, None, None] - px
        dy = p.uv[gg, 1][:, None, None] - py
        a, b, c = (p.conic[gg, k][:, None, None] for k in range(3))
        P = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
        alpha = np.minimum(0.99, p.opacity[gg][:, None, None] * np.exp(np.minimum(P, 0.0)))
        alpha = np.where((P <= 0) & inside, alpha, 0.0)
        out[s:s + 4096] = alpha.reshape(len(gg), -1).max(1)
    return out


@pytest.fixture
def sequential_walk():
    """The blends' one-CTA-per-tile walk: the split walk's chunks follow the list lengths, which
    culling changes, so only the sequential walk gives bit-identical results on both list kinds."""
    with _gpu.sequential_walk():
        yield


@pytest.mark.parametrize("which", ["cfg1", "multi", "low_opacity", "elongated"])
def test_culled_lists_keep_results(which, sequential_walk):
    w = _scene(which)
    rng = np.random.default_rng(35)
    n_pix = sum(c.W * c.H for c in w.cameras)
    dl = torch.as_tensor(rng.normal(0, 1, (n_pix, 4)), dtype=torch.float32, device="cuda").contiguous()
    r0, g0, eg0 = _run(w, False, dl)
    r1, g1, eg1 = _run(w, True, dl)
    assert r1.n_pairs < r0.n_pairs
    print(f"{which}: {r0.n_pairs} rectangle pairs -> {r1.n_pairs} after culling "
          f"({r1.n_pairs / max(r0.n_pairs, 1):.3f})")
    # unchanged results
    assert torch.equal(r0.rgba, r1.rgba)
    assert torch.equal(r0.final_T, r1.final_T)
    for v, c in enumerate(w.cameras):
        pix = np.stack(np.meshgrid(np.arange(c.W), np.arange(c.H)), -1).reshape(-1, 2)
        np.testing.assert_array_equal(_gpu.last_gaussian(r0, v, pix), _gpu.last_gaussian(r1, v, pix))
    # per-(tile, warp) gradient contributions are the same; only the order of the float atomics
    # that sum them differs: both meet the gradient bar against the FP64 oracle.
    ref = oracle.render(w.models, w.edits, w.cameras, bg=w.bg)
    excused = 0
    for v, c in enumerate(w.cameras):
        unc = _gpu.uncertain_records(ref.projs[v])
        extra = _gpu.uncertain_tile_mask(ref.projs[v], unc, c.W, c.H)
        err, exc, bad = _gpu.compare_image(r1.view_image(v).cpu().numpy(), ref.images[v], ref.margins[v], extra)
        assert bad == 0, (which, v, err)
        excused += exc
    assert excused <= max(3, 0.001 * r1.n_pix)
    dls = []
    for c in w.cameras:
        off = r0.cam_arr[len(dls)].pix_offset
        dls.append(dl[off:off + c.W * c.H].cpu().numpy().astype(np.float64).reshape(c.H, c.W, 4))
    gref = oracle.render_backward(ref, w.cameras, dls, bg=w.bg)
    for k in oracle.PARAMS:
        e0 = _gpu.assert_grad(g0[k].cpu().numpy(), gref.params[k], f"{k}, rectangle lists")
        e1 = _gpu.assert_grad(g1[k].cpu().numpy(), gref.params[k], f"{k}, culled lists")
        d01 = _gpu.rel_l2(g1[k].cpu().numpy().astype(np.float64), g0[k].cpu().numpy().astype(np.float64))
        print(f"{which} {k}: vs oracle (L2, element-wise) rect {e0[0]:.2e} {e0[1]:.2e} "
              f"culled {e1[0]:.2e} {e1[1]:.2e}; culled vs rect {d01:.2e}")
        if which != "elongated":
            assert d01 < 1e-4, (k, d01)
    ne = len(gref.edit)
    _gpu.assert_grad(eg0[:ne].cpu().numpy(), gref.edit, "edit table, rectangle lists")
    _gpu.assert_grad(eg1[:ne].cpu().numpy(), gref.edit, "edit table, culled lists")
    # culled lists: ordered sub-lists of the rectangle lists
    L0, L1 = _tile_lists(r0), _tile_lists(r1)
    comp = oracle.compose(w.models)
    tab = oracle.edit_table(w.edits)
    toff = np.cumsum([0] + [((c.W + 15) // 16) * ((c.H + 15) // 16) for c in w.cameras])
    drop_t, drop_g = [], []
    for t, (a, b) in enumerate(zip(L0, L1)):
        keep = np.isin(a, b)
        np.testing.assert_array_equal(a[keep], b)
        drop_t.append(np.full((~keep).sum(), t, np.int64))
        drop_g.append(a[~keep].astype(np.int64))
    drop_t, drop_g = np.concatenate(drop_t), np.concatenate(drop_g)
    assert len(drop_t) == r0.n_pairs - r1.n_pairs
    # every removed pair is skipped by the FP64 oracle at every pixel of its tile
    worst = 0.0
    for v, c in enumerate(w.cameras):
        sel = (drop_t >= toff[v]) & (drop_t < toff[v + 1])
        if not sel.any():
            continue
        p = oracle.project(comp, tab, c)
        lt = drop_t[sel] - toff[v]
        gx = (c.W + 15) // 16
        amax = _max_alpha_over_tile(p, c, drop_g[sel], lt % gx, lt // gx)
        worst = max(worst, float(amax.max()))
        assert (amax < ALPHA_MIN).all(), (v, float(amax.max()) * 255)
    print(f"{which}: largest FP64 alpha of a removed pair x 255 = {worst * 255:.4f}")


def test_culling_in_capacity_mode():
    """CAPACITY mode (no host sync) counts the same culled pairs and gives the same images."""
    w = sg.config1()
    rast, comp, table = _gpu.setup(w, cull=True)
    rast.forward(comp, table)
    torch.cuda.synchronize()
    n_exact = rast.n_pairs
    img = rast.rgba.clone()
    rast.forward(comp, table, mode="capacity")
    torch.cuda.synchronize()
    assert int(rast.d_n_pairs.item()) == n_exact
    assert torch.equal(rast.rgba, img)

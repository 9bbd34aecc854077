"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, small and ragged cases.

Rows: a1 compose/edit, a2 projection + shading, a3/a4 binning + radix sort (bit-exact on
shared inputs), a5 compositing (render-only on shared inputs, and end to end), a6/a7 backward.
Tolerances: images 2e-4 per channel outside oracle-certified near-ties; gradients 1e-3
relative L2 per tensor and 1e-3 of the tensor's largest entry element by element; keys,
values, ranges, radii and depth bits exact outside certified near-ties.
"""
import numpy as np
import pytest
import torch

import oracle
import scenegen as sg
from paper_2504_17954_gb300 import Rasterizer
from tests import _gpu

pytestmark = pytest.mark.gpu


def _multi_view_scene(seed=21, orbital=True):
    w = sg.tiny_scene(900, 48, 40, seed, log_scale_mu=-3.3, n_models=3)
    rng = np.random.default_rng(seed)
    sizes = [(48, 40), (37, 53), (64, 64)]
    cams = []
    for i, (W, H) in enumerate(sizes):
        hl = not (orbital and i % 2 == 1)
        cams.append(sg.look_at(3.0 * sg.random_direction(rng), W, H, headlight=hl,
                               light_dir=sg.orbital_light(20.0 + 10 * i, 0.3 * i)))
    ed = sg.random_edits(w.models, seed=seed)
    ed.lam = np.array([1.1, 0.9, 1.3, 0.7], np.float32)
    ed.bias = np.array([0.01, 0.0, -0.02, 2.0], np.float32)
    return sg.Workload("multi", w.models, cams, ed, bg=np.array([0.1, 0.05, 0.2], np.float32))


# ------------------------------------------------------------------ a1 + a2
@pytest.mark.parametrize("which", ["cfg1", "multi", "hidden"])
def test_project_matches_oracle(which):
    w = sg.config1() if which == "cfg1" else _multi_view_scene()
    if which == "hidden":
        w.edits.visible[1] = 0
    rast, comp, table = _gpu.setup(w)
    # a1: composition and edit table
    ref_comp = oracle.compose(w.models)
    for k in oracle.PARAMS:
        np.testing.assert_array_equal(getattr(comp, k).cpu().numpy().reshape(getattr(ref_comp, k).shape),
                                      getattr(ref_comp, k).astype(np.float32))
    np.testing.assert_array_equal(comp.model_id.cpu().numpy(), ref_comp.model_id)
    np.testing.assert_array_equal(table.cpu().numpy(), oracle.edit_table(w.edits).astype(np.float32))
    rast.project(comp, table)
    torch.cuda.synchronize()
    n = comp.n
    rad = rast.radius.cpu().numpy().reshape(len(w.cameras), n)
    xy = rast.xy.cpu().numpy().reshape(len(w.cameras), n, 2)
    co = rast.conic_o.cpu().numpy().reshape(len(w.cameras), n, 4)
    cd = rast.rgbd.cpu().numpy().reshape(len(w.cameras), n, 4)
    for v, cam in enumerate(w.cameras):
        p = oracle.project(ref_comp, oracle.edit_table(w.edits), cam)
        unc = _gpu.uncertain_records(p)
        mism = (rad[v] != p.radius) & ~unc
        assert not mism.any(), np.nonzero(mism)[0][:10]
        vis = (rad[v] > 0) & (p.radius > 0)
        assert vis.sum() > 0.5 * (p.radius > 0).sum()
        assert np.abs(xy[v][vis] - p.uv[vis]).max() < 2e-3
        # the record holds the conic in completed-square form (g, b, c), g = a - b^2/c = 1/Sigma'_xx
        want = np.c_[1.0 / p.cov[vis, 0], p.conic[vis, 1:]]
        cmax = np.abs(p.conic[vis]).max(1, keepdims=True)
        assert (np.abs(co[v][vis, :3] - want) / cmax).max() < 1e-4
        assert np.abs(co[v][vis, 3] - p.opacity[vis]).max() < 1e-6
        assert np.abs(cd[v][vis, :3] - p.rgb[vis]).max() < 1e-5
        # depth: the float64 camera z rounded once to float32, the same bits on both sides
        # except where z lies within 2^-40 (relative) of a rounding midpoint (certified, counted)
        dok = vis & ~_gpu.depth_uncertain(p)
        np.testing.assert_array_equal(cd[v][dok, 3].view(np.uint32), p.depth[dok].astype(np.float32).view(np.uint32))
        print(f"{which} view {v}: {int(vis.sum())} depth keys compared, "
              f"{int((vis & _gpu.depth_uncertain(p)).sum())} certified near a float32 rounding midpoint")


# ------------------------------------------------------------------ a3 + a4 (shared inputs, bit-exact)
def _gpu_bin_from(sizes, xy, rad, depth, mode="exact", capacity=None):
    V, n = rad.shape
    cams = [sg.look_at([3, 0, 0], W, H) for (W, H) in sizes]
    rast = Rasterizer(cams, n, 1, capacity=capacity, cull=False)  # the rectangle lists
    rast.xy.copy_(torch.as_tensor(xy.reshape(-1, 2)))
    rast.radius.copy_(torch.as_tensor(rad.reshape(-1)))
    d = np.zeros((V * n, 4), np.float32)
    d[:, 3] = depth.reshape(-1)
    rast.rgbd.copy_(torch.as_tensor(d))
    if mode == "exact":
        rast.bin("exact")
    else:
        rast.bin("capacity")
        torch.cuda.synchronize()
        rast.n_pairs = int(rast.d_n_pairs.item())
    torch.cuda.synchronize()
    return rast


@pytest.fixture(params=[(0, 0), (0, 1), (1, 0)], ids=["lookback", "lookback_early", "rts"])
def sort_scan(request):
    from paper_2504_17954_gb300 import _native as N
    names = ("sort_scan", "sort_early")
    old = [N.ivrgs_get_option(k) for k in names]
    for k, v in zip(names, request.param):
        N.ivrgs_set_option(k, v)
    yield request.param
    for k, v in zip(names, old):
        N.ivrgs_set_option(k, v)


@pytest.mark.parametrize("case", ["small", "ties", "ragged", "many", "dense1", "dense2", "single_tile", "empty"])
@pytest.mark.parametrize("mode", ["exact", "capacity"])
def test_bin_bit_exact(case, mode, sort_scan):
    if case == "small":
        sizes, n, seed, kw = [(64, 48)], 500, 1, {}
    elif case == "ties":
        sizes, n, seed, kw = [(128, 96), (96, 128)], 3000, 2, {"tie_frac": 0.9}
    elif case == "ragged":
        sizes, n, seed, kw = [(37, 53), (100, 7), (16, 16), (250, 130)], 2000, 3, {}
    elif case == "many":
        sizes, n, seed, kw = [(512, 512), (800, 800), (1024, 768)], 60000, 4, {"max_radius": 60}
    elif case == "dense1":  # 12 tiles (one radix pass), each run spread over several radix tiles
        sizes, n, seed, kw = [(64, 48)], 80000, 10, {"max_radius": 40}
    elif case == "dense2":  # 289 tiles (two passes), runs of thousands of pairs
        sizes, n, seed, kw = [(272, 272)], 40000, 11, {"max_radius": 150}
    elif case == "single_tile":
        sizes, n, seed, kw = [(16, 16)], 5000, 5, {}
    else:
        sizes, n, seed, kw = [(64, 64)], 100, 6, {}
    xy, rad, depth = sg.synthetic_projected(sizes, n, seed, **kw)
    if case == "empty":
        rad[:] = 0
    ref = oracle.bin_pairs(xy, rad, depth, sizes)
    cap = None if mode == "exact" else len(ref.keys) + 12345
    rast = _gpu_bin_from(sizes, xy, rad, depth, mode, cap)
    assert rast.n_pairs == len(ref.keys)
    k, v, r = _gpu.gpu_keys(rast)
    np.testing.assert_array_equal(k, ref.keys)
    np.testing.assert_array_equal(v, ref.values)
    np.testing.assert_array_equal(r, ref.ranges)
    if case == "many":
        assert len(ref.keys) > 20 * 3072  # several radix tiles and all passes exercised
    if case.startswith("dense"):
        assert (r[:, 1] - r[:, 0]).max() > 2 * 4096  # a run covering three radix tiles or more


def test_bin_capacity_reporting():
    sizes = [(256, 256)]
    xy, rad, depth = sg.synthetic_projected(sizes, 4000, 7)
    ref = oracle.bin_pairs(xy, rad, depth, sizes)
    # exact mode grows to fit; capacity mode reports the true count in d_n_pairs
    small = len(ref.keys) // 3
    rast = _gpu_bin_from(sizes, xy, rad, depth, "capacity", small)
    assert rast.n_pairs == len(ref.keys) > rast.capacity
    rast2 = _gpu_bin_from(sizes, xy, rad, depth, "exact", small)
    assert rast2.n_pairs == len(ref.keys)
    k, v, r = _gpu.gpu_keys(rast2)
    np.testing.assert_array_equal(k, ref.keys)


# ------------------------------------------------------------------ a5 render-only on shared inputs
def _shared_records(w):
    """Oracle float64 projection rounded to float32: the same inputs for both blends. The
    conic travels as the record's (g, b, c) (g = 1/Sigma'_xx) rounded to float32 (held in the
    returned records' `cov` field); the oracle blends the conic those values define,
    a = g + b^2/c."""
    comp = oracle.compose(w.models)
    tab = oracle.edit_table(w.edits)
    projs = [oracle.project(comp, tab, c) for c in w.cameras]
    f32 = []
    for p in projs:
        live = p.radius > 0
        g32 = np.where(live, 1.0 / np.where(live, p.cov[:, 0], 1.0), 1.0).astype(np.float32).astype(np.float64)
        b32, c32 = (p.conic[:, k].astype(np.float32).astype(np.float64) for k in (1, 2))
        c32 = np.where(live, c32, 1.0)
        q = oracle.Projected(uv=p.uv.astype(np.float32).astype(np.float64),
                             cov=np.c_[g32, b32, c32], conic=np.c_[g32 + b32 * b32 / c32, b32, c32],
                             opacity=p.opacity.astype(np.float32).astype(np.float64),
                             rgb=p.rgb.astype(np.float32).astype(np.float64),
                             depth=p.depth.astype(np.float32).astype(np.float64), radius=p.radius,
                             radius_margin=p.radius_margin)
        f32.append(q)
    return f32


@pytest.mark.parametrize("which", ["cfg1", "multi"])
def test_render_only_matches_oracle_on_shared_records(which):
    w = sg.config1() if which == "cfg1" else _multi_view_scene(seed=23)
    projs = _shared_records(w)
    sizes = [(c.W, c.H) for c in w.cameras]
    n = projs[0].radius.shape[0]
    rast = Rasterizer(w.cameras, n, len(w.models), bg=w.bg, cull=False)  # lists compared with the oracle's
    rast.xy.copy_(torch.as_tensor(np.concatenate([p.uv for p in projs]).astype(np.float32)))
    rast.conic_o.copy_(torch.as_tensor(np.concatenate(  # the record form (g, b, c, o')
        [np.c_[p.cov, p.opacity] for p in projs]).astype(np.float32)))
    rast.rgbd.copy_(torch.as_tensor(np.concatenate([np.c_[p.rgb, p.depth] for p in projs]).astype(np.float32)))
    rast.radius.copy_(torch.as_tensor(np.concatenate([p.radius for p in projs]).astype(np.int32)))
    rast.bin("exact")
    rast.render()
    torch.cuda.synchronize()
    bins = oracle.bin_pairs(*oracle.decision_inputs(projs), sizes)
    k, vals, r = _gpu.gpu_keys(rast)
    np.testing.assert_array_equal(k, bins.keys)
    bg = np.asarray(w.bg, np.float64)
    total_excused = 0
    for v, (c, p) in enumerate(zip(w.cameras, projs)):
        rgba = np.zeros((c.H, c.W, 4)); T = np.zeros((c.H, c.W)); last = np.zeros((c.H, c.W), np.uint32)
        mg = np.zeros((c.H, c.W, oracle.N_MARGINS))
        oracle.lib().orc_render_view(*[oracle._p(a) for a in (p.uv, p.conic, p.opacity, p.rgb)],
                                     oracle._p(bins.values, oracle.C.c_uint32), oracle._p(bins.ranges, oracle.C.c_uint32),
                                     oracle.C.c_int64(int(bins.tile_offset[v])), oracle.C.c_int32(c.W),
                                     oracle.C.c_int32(c.H), oracle.C.c_int32(16), oracle.C.c_int32(16),
                                     oracle._p(np.ascontiguousarray(bg)), oracle._p(rgba), oracle._p(T),
                                     oracle._p(last, oracle.C.c_uint32), oracle._p(mg))
        gimg = rast.view_image(v).cpu().numpy()
        err, excused, bad = _gpu.compare_image(gimg, rgba, mg)
        assert bad == 0, (v, err)
        total_excused += excused
        glast = rast.view_image(v, rast.last).cpu().numpy()
        ok = ~_gpu.near_tie(mg)
        np.testing.assert_array_equal(glast[ok], last[ok].astype(np.int32))
        np.testing.assert_allclose(rast.view_image(v, rast.final_T).cpu().numpy()[ok], T[ok], rtol=2e-4, atol=1e-6)
    assert total_excused <= max(3, 0.001 * rast.n_pix)


# ------------------------------------------------------------------ end to end forward
# blend launch shapes: (pixels per thread, render_split (0 = split by tile count, the default,
# which splits the small scenes here (few tiles) at 256 entries; 2 = one CTA per tile; 1 = split
# always; 4 = long runs first), entries per chunk). "split32" cuts every run longer than 32
# entries into up to 8 chunks over a CTA cluster, "longfirst32" walks the runs longer than 32
# entries in a launch of their own, first.
@pytest.fixture(params=[(0, 0, 256), (1, 2, 384), (2, 2, 384), (4, 2, 384), (8, 2, 384), (0, 2, 384), (0, 1, 32),
                        (4, 1, 32), (1, 1, 32), (0, 4, 32)],
                ids=["ppt_auto", "ppt1", "ppt2", "ppt4", "ppt8", "nosplit", "split32", "split32_ppt4", "split32_ppt1",
                     "longfirst32"])
def pixels_per_thread(request):
    from paper_2504_17954_gb300 import _native as N
    names = ("render_pixels_per_thread", "render_bwd_pixels_per_thread", "render_split", "render_split_min")
    old = [N.ivrgs_get_option(k) for k in names]
    ppt, split, smin = request.param
    for k, val in zip(names, (ppt, ppt, split, smin)):
        N.ivrgs_set_option(k, val)
    yield request.param
    for k, val in zip(names, old):
        N.ivrgs_set_option(k, val)


@pytest.mark.parametrize("which", ["cfg1", "multi"])
def test_forward_end_to_end(which, pixels_per_thread):
    w = sg.config1() if which == "cfg1" else _multi_view_scene(seed=25)
    rast, comp, table = _gpu.setup(w, cull=False)  # tile lists compared with the oracle's
    rast.forward(comp, table)
    torch.cuda.synchronize()
    ref = oracle.render(w.models, w.edits, w.cameras, bg=w.bg)
    # tile lists: identical after removing certified-uncertain records
    k, vals, r = _gpu.gpu_keys(rast)
    n = comp.n
    unc_all = [_gpu.uncertain_records(p) for p in ref.projs]
    view_of = lambda keys: np.searchsorted(ref.bins.tile_offset, (keys >> np.uint64(32)).astype(np.int64),
                                           side="right") - 1
    def strip(keys, values):
        vv = view_of(keys)
        keep = np.array([not unc_all[a][b] for a, b in zip(vv, values)], bool) if len(keys) else np.zeros(0, bool)
        return keys[keep], values[keep]
    gk, gv = strip(k, vals)
    ok_, ov = strip(ref.bins.keys, ref.bins.values)
    np.testing.assert_array_equal(gk, ok_)
    np.testing.assert_array_equal(gv, ov)
    total_excused = 0
    for v, c in enumerate(w.cameras):
        extra = _gpu.uncertain_tile_mask(ref.projs[v], unc_all[v], c.W, c.H)
        err, excused, bad = _gpu.compare_image(rast.view_image(v).cpu().numpy(), ref.images[v], ref.margins[v], extra)
        assert bad == 0, (v, err)
        total_excused += excused
    assert total_excused <= max(3, 0.001 * rast.n_pix)


# ------------------------------------------------------------------ backward
@pytest.mark.parametrize("which", ["fd", "fd_orbital", "fd_table_light", "multi"])
def test_backward_matches_oracle(which, pixels_per_thread):
    if which.startswith("fd"):
        from tests.test_oracle_grad_fd import _scene
        models, ed, cams = _scene(which != "fd", which == "fd_table_light")
        w = sg.Workload("fd", models, cams, ed, bg=np.array([0.2, 0.1, 0.3], np.float32))
    else:
        w = _multi_view_scene(seed=27)
    rast, comp, table = _gpu.setup(w)
    rast.forward(comp, table)
    rng = np.random.default_rng(4)
    dls = [rng.normal(0, 1, (c.H, c.W, 4)) for c in w.cameras]
    dl = torch.as_tensor(np.concatenate([d.reshape(-1, 4) for d in dls]), dtype=torch.float32, device="cuda")
    grad, egrad = rast.backward(comp, table, dl.contiguous())
    torch.cuda.synchronize()
    ref = oracle.render(w.models, w.edits, w.cameras, bg=w.bg)
    gref = oracle.render_backward(ref, w.cameras, dls, bg=w.bg)
    for k in oracle.PARAMS:
        _gpu.assert_grad(getattr(grad, k).cpu().numpy(), gref.params[k], k)
    ne = len(gref.edit)
    eg = egrad.cpu().numpy().astype(np.float64)
    M = len(w.models)
    for m in range(M):
        sl = slice(8 * m, 8 * m + 4)
        _gpu.assert_grad(eg[sl], gref.edit[sl], f"edit of model {m}")
    _gpu.assert_grad(eg[8 * M:ne], gref.edit[8 * M:], "lambda, b and the global light")
    if which == "fd_table_light":  # the global light's gradient on its own
        _gpu.assert_grad(eg[8 * M + 8:8 * M + 11], gref.edit[8 * M + 8:8 * M + 11], "global light")
        assert np.abs(gref.edit[8 * M + 8:8 * M + 11]).max() > 0
    light = eg[ne:].reshape(len(w.cameras), 4)[:, :3]
    for v, c in enumerate(w.cameras):
        if c.headlight:
            assert np.all(light[v] == 0)
        else:
            _gpu.assert_grad(light[v], gref.light[v], f"light of view {v}")

"""The blends' results do not depend on their launch shape. At 1, 2, 4 and 8 pixels per thread
(the one-pixel walks take several list entries per step, the others one) the forward gives every
pixel the same colour, final transmittance and last contributor bit for bit: each pixel sees the
same operations in the same order, only the thread that holds it changes. The same at 16 x 8
tiles (1, 2 and 4 pixels per thread). Sequential walk: the split walk regroups the products by
chunk. The backward's gradients at 1 and 4 pixels per thread agree up to the order of the float32
sums (each thread adds its own pixels first, then the warp and the atomics add across threads)."""
import numpy as np
import pytest
import torch

import oracle
import scenegen as sg
from tests import _gpu
from tests.test_gpu_parity import _multi_view_scene

pytestmark = pytest.mark.gpu

_PPT = ("render_pixels_per_thread", "render_bwd_pixels_per_thread")


def _scene(which):
    if which == "cfg1":
        return sg.config1()
    if which == "multi":
        return _multi_view_scene(seed=41)
    # long runs: 20,000 Gaussians over one 64 x 48 view, a few thousand entries per tile, so that
    # the walks span several staged batches, pixels terminate inside a batch and the one-pixel
    # walks meet every remainder of a batch's list modulo their entries per step
    w = sg.tiny_scene(20000, 64, 48, 43, log_scale_mu=-2.6)
    return sg.Workload("long_runs", w.models, w.cameras, w.edits, bg=np.array([0.3, 0.2, 0.1], np.float32))


def _run(w, ppt, tile_h, dl=None):
    from paper_2504_17954_gb300 import _native as N
    old = [N.ivrgs_get_option(k) for k in _PPT]
    for k in _PPT:
        N.ivrgs_set_option(k, ppt)
    try:
        with _gpu.sequential_walk():
            rast, comp, table = _gpu.setup(w, tile_h=tile_h)
            rast.forward(comp, table)
            grads = None
            if dl is not None:
                g, eg = rast.backward(comp, table, dl)
                grads = {k: getattr(g, k).detach().cpu().numpy() for k in oracle.PARAMS}
                grads["edit"] = eg.cpu().numpy()
            torch.cuda.synchronize()
            return rast.rgba.clone(), rast.final_T.clone(), rast.last.clone(), rast.n_pairs, grads
    finally:
        for k, v in zip(_PPT, old):
            N.ivrgs_set_option(k, v)


@pytest.mark.parametrize("tile_h", [16, 8])
@pytest.mark.parametrize("which", ["cfg1", "multi", "long_runs"])
def test_forward_bits_do_not_depend_on_pixels_per_thread(which, tile_h):
    w = _scene(which)
    shapes = (1, 2, 4, 8) if tile_h == 16 else (1, 2, 4)
    ref = _run(w, 4, tile_h)
    assert ref[3] > 0
    for ppt in shapes:
        if ppt == 4:
            continue
        out = _run(w, ppt, tile_h)
        assert out[3] == ref[3]
        assert torch.equal(out[0], ref[0]), (which, tile_h, ppt)
        assert torch.equal(out[1], ref[1]), (which, tile_h, ppt)
        assert torch.equal(out[2], ref[2]), (which, tile_h, ppt)


@pytest.mark.parametrize("which", ["multi", "long_runs"])
def test_backward_at_one_and_four_pixels_per_thread(which):
    w = _scene(which)
    n_pix = sum(c.W * c.H for c in w.cameras)
    rng = np.random.default_rng(45)
    dl = torch.as_tensor(rng.normal(0, 1, (n_pix, 4)), dtype=torch.float32, device="cuda").contiguous()
    g4 = _run(w, 4, 16, dl)[4]
    g1 = _run(w, 1, 16, dl)[4]
    for k, ref in g4.items():
        scale = max(float(np.abs(ref).max()), 1e-30)
        err = float(np.abs(g1[k] - ref).max()) / scale
        assert err <= 1e-4, (k, err)

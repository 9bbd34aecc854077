"""The CUDA path against the stored regression record ``tests/golden/oracle_two_models_40x24.json``
(two basic models with palette, opacity and light-magnitude edits; a headlight and an orbital
view of 40 x 24 pixels), through the C ABI, without running the oracle:

* tile lists (rectangle mode) bit for bit: the record holds no record at a float32 decision
  tie, which its writer checks;
* sampled pixels within 2e-4 and their last contributors exactly, skipping the pixels the
  record flags as near a decision tie (none at present);
* per-channel image sums within 2e-4 per pixel;
* the reverse mode for the record's closed-form dL/dRGBA: attribute, edit and light
  gradients within 1e-3 (relative L2, and element by element of the largest entry), as the
  other parity tests.
"""
import importlib.util
import json
import os

import numpy as np
import pytest
import torch

import oracle
from tests import _gpu

pytestmark = pytest.mark.gpu

_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
_spec = importlib.util.spec_from_file_location("make_golden", os.path.join(_DIR, "make_golden.py"))
mg = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(mg)


def test_cuda_path_matches_the_record():
    with open(os.path.join(_DIR, mg.NAME)) as f:
        rec = json.load(f)
    out = rec["outputs"]
    w = mg.workload_from(rec["inputs"])
    rast, comp, table = _gpu.setup(w, cull=False)
    rgba = rast.forward(comp, table).clone()
    torch.cuda.synchronize()

    _, vals, ranges = _gpu.gpu_keys(rast)
    np.testing.assert_array_equal(vals.astype(np.int64), np.asarray(out["values"], np.int64))
    want_r = np.asarray(out["ranges"], np.int64)
    np.testing.assert_array_equal(ranges[:len(want_r)].astype(np.int64), want_r)

    for v, c in enumerate(w.cameras):
        rv = out["views"][v]
        img = rast.view_image(v, rgba).cpu().numpy().astype(np.float64).reshape(-1, 4)
        last = rast.view_image(v, rast.last).cpu().numpy().reshape(-1)
        pix = np.asarray(rv["pixels"])
        ok = ~np.asarray(rv["near_tie"], bool)
        err = np.abs(img[pix] - np.asarray(rv["rgba"])).max(1)
        assert float(err[ok].max()) <= _gpu.IMG_TOL, (v, float(err[ok].max()))
        np.testing.assert_array_equal(last[pix][ok], np.asarray(rv["last"])[ok])
        assert np.all(np.abs(img.sum(0) - np.asarray(rv["rgba_sum"])) <= _gpu.IMG_TOL * c.W * c.H), v

    dl = torch.as_tensor(np.concatenate([mg.dl_drgba(c.W, c.H, v).reshape(-1, 4) for v, c in enumerate(w.cameras)]),
                         dtype=torch.float32, device="cuda").contiguous()
    grad, egrad = rast.backward(comp, table, dl)
    torch.cuda.synchronize()
    for k in oracle.PARAMS:
        want = np.asarray(out["grad"][k], np.float64)
        got = getattr(grad, k).cpu().numpy().astype(np.float64).reshape(want.shape)
        _gpu.assert_grad(got, want, k)
    eg = egrad.cpu().numpy().astype(np.float64)
    want_e = np.asarray(out["grad_edit"], np.float64)
    M = len(w.models)
    for m in range(M):
        sl = slice(8 * m, 8 * m + 4)
        _gpu.assert_grad(eg[sl], want_e[sl], f"edit of model {m}")
    _gpu.assert_grad(eg[8 * M:8 * M + 8], want_e[8 * M:8 * M + 8], "lambda and b")
    light = eg[len(want_e):].reshape(len(w.cameras), 4)[:, :3]
    want_l = np.asarray(out["grad_light"], np.float64)
    assert np.all(light[0] == 0)  # the headlight view has no light direction to move
    _gpu.assert_grad(light[1], want_l[1], "light of view 1")

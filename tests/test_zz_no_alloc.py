"""ivrgs_render_backward_static: the backward for callers that cannot call cudaMalloc.

Such callers (a plugin inside a host application that owns the device memory, an interactive
loop that must not stall on an allocation) get the same gradients without passing a workspace:
the scratch is a fixed device array inside the library. This test calls it through the C ABI
twice in a row and checks both results against ivrgs_render_backward with a caller-provided
workspace, at the gradient tolerance of the parity tests (1e-3 relative L2 per tensor), and
that an oversized request is refused up front. Collected last on purpose (file name).
"""
import ctypes as C

import numpy as np
import pytest
import torch

import scenegen as sg
from paper_2504_17954_gb300 import _native as N
from paper_2504_17954_gb300.rasterizer import ATTRS, Gaussians, _stream, _vp
from tests import _gpu

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3


def _backward_static(rast, comp, table, dl):
    grad = Gaussians.empty(rast.n, rast.n_models, rast.device)
    grad.model_id = None
    egrad = torch.empty_like(rast.edit_grad)
    gs, gr = comp.struct(), grad.struct()
    p, b = rast.projected_struct(), rast.bins_struct()
    N.ivrgs_render_backward_static(C.byref(gs), _vp(table), C.byref(p), C.byref(b), rast.cam_arr, rast.V,
                                   rast.lowpass, rast.bg, _vp(rast.final_T), _vp(rast.last), _vp(dl),
                                   C.byref(gr), _vp(egrad), _stream())
    return grad, egrad


def test_static_scratch_backward_matches_workspace_backward_twice():
    w = sg.config1()
    w.bg = np.array([0.1, 0.2, 0.3], np.float32)
    rast, comp, table = _gpu.setup(w)
    assert rast.n * rast.V * 36 + 256 <= N.IVRGS_STATIC_SCRATCH_BYTES
    rast.forward(comp, table)
    dl = torch.as_tensor(np.random.default_rng(4).normal(0, 1, (rast.n_pix, 4)), dtype=torch.float32,
                         device="cuda").contiguous()
    ref, eref = rast.backward(comp, table, dl)
    ref = {k: getattr(ref, k).detach().cpu().numpy().astype(np.float64) for k in ATTRS}
    eref = eref.detach().cpu().numpy().astype(np.float64)
    assert np.linalg.norm(ref["mean"]) > 0
    for _ in range(2):
        grad, egrad = _backward_static(rast, comp, table, dl)
        torch.cuda.synchronize()
        for k in ATTRS:
            _gpu.assert_grad(getattr(grad, k).cpu().numpy(), ref[k], k, GRAD_TOL)
        _gpu.assert_grad(egrad.cpu().numpy(), eref, "edit table", GRAD_TOL)


def test_static_scratch_refuses_oversized_problems():
    g = N.ivrgs_gaussians()
    g.n = 10_000_000
    g.n_models = 1
    cams = (N.ivrgs_camera * 1)()
    st = N.lib().ivrgs_render_backward_static(C.byref(g), None, None, None, cams, 1, 0.3, None, None, None, None,
                                              None, None, None)
    assert st == N.IVRGS_ERR_CAPACITY
    assert "scratch" in N.last_error()

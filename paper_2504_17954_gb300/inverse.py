"""Inverse volume exploration (Sec. 4.6): fit the edits of a composed model to a reference image.

All Gaussian attributes stay fixed. The learnable values are the edit table's per-model palette
colour c_p and opacity scale, the global lambda and b, and (orbital light, with the table's
global light switched on) the light direction as polar and azimuthal angles. One iteration is
projection + binning + compositing, the image loss (ivrgs_image_loss: (1 - l) L1 + l (1 - SSIM)),
the backward (edit gradients; the per-Gaussian gradients are computed too and discarded) and an
Adam step on the edit table (ivrgs_edit_adam); every step runs in the library's kernels and the
whole iteration can be captured into one CUDA graph. This module only marshals arguments.
"""
from __future__ import annotations

from typing import List

import torch

from . import _native as N
from .rasterizer import Gaussians, Rasterizer, _stream, _vp

LEARN_ALL = (N.IVRGS_LEARN_COLOR | N.IVRGS_LEARN_OPACITY | N.IVRGS_LEARN_LIGHT_MAGNITUDE |
             N.IVRGS_LEARN_LIGHT_DIRECTION)


class InverseExplorer:
    """``rast`` renders the reference views; ``target`` holds the reference images packed like
    ``rast.rgba`` ([n_pix, 4], alpha ignored); ``edit_table`` is updated in place."""

    def __init__(self, rast: Rasterizer, g: Gaussians, edit_table: torch.Tensor, target: torch.Tensor,
                 learn: int = LEARN_ALL, lr: float = 0.01, lambda_ssim: float = 0.2,
                 betas=(0.9, 0.999), eps: float = 1e-8):
        if target.shape != rast.rgba.shape or target.dtype != torch.float32 or not target.is_contiguous():
            raise ValueError("target must be a contiguous float32 tensor shaped like rast.rgba")
        self.rast, self.g, self.table, self.target = rast, g, edit_table, target
        self.M = rast.n_models
        self.learn, self.lr, self.lam = int(learn), float(lr), float(lambda_ssim)
        self.b1, self.b2, self.eps = float(betas[0]), float(betas[1]), float(eps)
        dev = rast.device
        self.ws_loss_bytes = N.ivrgs_image_loss_workspace(rast.cam_arr, rast.V)
        self.ws_loss = torch.empty(self.ws_loss_bytes, dtype=torch.uint8, device=dev)
        self.loss = torch.zeros(3, dtype=torch.float32, device=dev)  # (loss, L1, SSIM)
        self.dL = torch.zeros_like(rast.rgba)
        self.grad = Gaussians.empty(rast.n, self.M, dev)
        self.grad.model_id = None
        self.state = torch.empty(N.lib().ivrgs_edit_adam_state_floats(self.M), dtype=torch.float32, device=dev)
        N.ivrgs_edit_adam_init(_vp(edit_table), self.M, _vp(self.state), _stream())
        self.graph = None

    def _loss(self, stream=None):
        N.ivrgs_image_loss(_vp(self.rast.rgba), _vp(self.target), self.rast.cam_arr, self.rast.V, self.lam,
                           _vp(self.ws_loss), self.ws_loss_bytes, _vp(self.loss), _vp(self.dL), _stream(stream))

    def _adam(self, stream=None):
        N.ivrgs_edit_adam(_vp(self.table), _vp(self.rast.edit_grad), self.M, _vp(self.state), self.learn, self.lr,
                          self.b1, self.b2, self.eps, _stream(stream))

    def _iteration(self, mode: str, adam: bool = True, stream=None):
        self.rast.forward(self.g, self.table, mode=mode, stream=stream)
        self._loss(stream)
        self.rast.backward(self.g, self.table, self.dL, grad=self.grad, stream=stream)
        if adam:
            self._adam(stream)

    def step(self):
        """One iteration (eager, EXACT-mode binning)."""
        self._iteration("exact")

    def capture(self, warmup: int = 2) -> "torch.cuda.CUDAGraph":
        """Capture one iteration (CAPACITY-mode binning) as a CUDA graph; the warm-up runs the
        iteration without its optimiser step, so the parameters are unchanged."""
        self.rast.forward(self.g, self.table, mode="exact")
        cap = self.rast.capacity
        self.rast._ensure_capacity(int(self.rast.n_pairs * 1.5) + 4096)
        if self.rast.capacity != cap:
            self.rast.forward(self.g, self.table, mode="exact")
        N.prof_enable(False)
        side = torch.cuda.Stream(device=self.rast.device)
        side.wait_stream(torch.cuda.current_stream(self.rast.device))
        with torch.cuda.stream(side):
            for _ in range(warmup):
                self._iteration("capacity", adam=False)
        torch.cuda.current_stream(self.rast.device).wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self._iteration("capacity")
        self.graph = graph
        return graph

    def overflowed(self) -> bool:
        """True if the last CAPACITY-mode binning had more pairs than the buffer holds."""
        return int(self.rast.d_n_pairs.item()) > self.rast.capacity

    def run(self, iters: int, graph: bool = True, record_every: int = 0) -> List[float]:
        """Run ``iters`` iterations; returns the loss recorded every ``record_every`` iterations
        (a device-to-host read each time; 0 = only the last)."""
        hist: List[float] = []
        if graph and self.graph is None:
            self.capture()
        for k in range(iters):
            if graph:
                self.graph.replay()
            else:
                self.step()
            if record_every and (k + 1) % record_every == 0:
                hist.append(float(self.loss[0].item()))
        if graph and self.overflowed():
            raise RuntimeError("pair buffer overflowed during graph replay; capture again")
        hist.append(float(self.loss[0].item()))
        return hist

    def step_count(self) -> int:
        return int(self.state[-1].item())

    def light_angles(self):
        P = 4 * self.M + 10
        return float(self.state[2 * P].item()), float(self.state[2 * P + 1].item())

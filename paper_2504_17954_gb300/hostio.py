"""Forward + backward steps on Gaussians held in pinned host memory, with the transfers of
neighbouring steps overlapping the compute.

Each step copies its float32 attributes in (one block, see ``HOST_LAYOUT``), renders the
cameras of a Rasterizer, runs the reverse mode for a given dL/dRGBA, and copies the image and
the attribute gradients back. Three CUDA streams carry the work: host->device copies, compute,
device->host copies. The inputs and the gradients have two device slots each, so step i+1's
attributes arrive while step i computes, and step i's gradients leave while step i+1 computes;
the image of step i leaves during step i's backward. Every step still moves all of its own
bytes: only the waiting between copy and compute is removed. The compute of each slot is
replayed from two CUDA graphs (forward, backward), captured once, so a step costs a handful of
launches instead of one per kernel.
"""
from __future__ import annotations

from typing import List, Sequence

import torch

from . import _native as N
from .rasterizer import ATTRS, WIDTH, Gaussians, Rasterizer

# order and widths of the attribute arrays inside one host (or device) block of 21 n floats
HOST_LAYOUT = tuple((k, WIDTH[k]) for k in ATTRS)
FLOATS_PER_GAUSSIAN = sum(w for _, w in HOST_LAYOUT)


def block_views(block: torch.Tensor, n: int) -> List[torch.Tensor]:
    """The attribute arrays inside a block of FLOATS_PER_GAUSSIAN * n floats, in ATTRS order:
    [n, 3] mean, [n, 3] log_scale, [n, 4] quat, [n] opacity_logit, [n, 3] dcolor, [n, 3] normal,
    [n, 4] kads (each array contiguous, one after the other)."""
    out, o = [], 0
    for _, w in HOST_LAYOUT:
        t = block[o:o + w * n]
        out.append(t.view(n, w) if w > 1 else t)
        o += w * n
    return out


def pack_host(g: Gaussians) -> torch.Tensor:
    """A pinned host block holding the float32 attributes of g (the input of one step). The
    pipeline carries the Blinn-Phong attribute set; SH colour is not part of the block."""
    if g.precision != N.IVRGS_FP32:
        raise ValueError("the host pipeline carries float32 attributes")
    if g.sh is not None:
        raise ValueError("the host pipeline carries the Blinn-Phong attributes, not SH colour")
    n = g.n
    blk = torch.empty(FLOATS_PER_GAUSSIAN * n, dtype=torch.float32).pin_memory()
    for t, k in zip(block_views(blk, n), ATTRS):
        t.copy_(getattr(g, k).reshape(t.shape))
    return blk


class HostPipeline:
    """Steps of forward + backward over host-resident float32 Gaussians (one Rasterizer, one
    model-id array shared by all steps). ``edit_table`` and ``dL_drgba`` are device tensors read
    by every step: change their contents between calls, not the tensors themselves (the
    captured graphs hold their addresses). The Rasterizer's pair buffer must already be sized
    (one exact-mode forward) with room for the steps' pairs."""

    def __init__(self, rast: Rasterizer, model_id: torch.Tensor, n_models: int, edit_table: torch.Tensor,
                 dL_drgba: torch.Tensor, graphs: bool = True):
        self.rast = rast
        n = rast.n
        dev = rast.device
        self.n = n
        self.model_id = model_id
        self.n_models = n_models
        self.table = edit_table
        self.dL = dL_drgba
        self.d_in = [torch.empty(FLOATS_PER_GAUSSIAN * n, dtype=torch.float32, device=dev) for _ in range(2)]
        self.d_grad = [torch.empty(FLOATS_PER_GAUSSIAN * n, dtype=torch.float32, device=dev) for _ in range(2)]
        self.s_in = torch.cuda.Stream(device=dev)
        self.s_comp = torch.cuda.Stream(device=dev)
        self.s_out = torch.cuda.Stream(device=dev)
        self.h2d_bytes = FLOATS_PER_GAUSSIAN * n * 4
        self.d2h_bytes = rast.n_pix * 16 + FLOATS_PER_GAUSSIAN * n * 4
        self.graphs = self._capture() if graphs else None

    def _fwd(self, s: int):
        self.rast.forward(self._gaussians(self.d_in[s]), self.table, mode="capacity")

    def _bwd(self, s: int):
        self.rast.backward(self._gaussians(self.d_in[s]), self.table, self.dL,
                           grad=self._gaussians(self.d_grad[s], False))

    def _capture(self):
        """Forward and backward graphs for both slots, captured on the compute stream after a
        warm-up there (the slots' contents do not matter to the capture)."""
        rast = self.rast
        if rast.ws_bwd is None:
            rast.ws_bwd = torch.empty(rast.ws_bwd_bytes, dtype=torch.uint8, device=rast.device)
        N.prof_enable(False)
        for t in self.d_in + self.d_grad:
            t.zero_()
        self.s_comp.wait_stream(torch.cuda.current_stream(rast.device))
        with torch.cuda.stream(self.s_comp):
            for s in range(2):
                self._fwd(s)
                self._bwd(s)
        torch.cuda.current_stream(rast.device).wait_stream(self.s_comp)
        out = []
        for s in range(2):
            gf, gb = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
            with torch.cuda.graph(gf, stream=self.s_comp):
                self._fwd(s)
            with torch.cuda.graph(gb, stream=self.s_comp):
                self._bwd(s)
            out.append((gf, gb))
        return out

    def _gaussians(self, block: torch.Tensor, with_ids: bool = True) -> Gaussians:
        return Gaussians(*block_views(block, self.n), model_id=self.model_id if with_ids else None,
                         n_models=self.n_models)

    def run(self, host_in: Sequence[torch.Tensor], host_img: Sequence[torch.Tensor],
            host_grad: Sequence[torch.Tensor]):
        """Step i reads host_in[i] and writes host_img[i] ([n_pix, 4]) and host_grad[i] (a block
        like the input); all host tensors pinned. Work is queued behind the current stream and
        the current stream waits for all of it, so events recorded around the call time the
        whole transfer."""
        rast = self.rast
        cur = torch.cuda.current_stream(rast.device)
        for s in (self.s_in, self.s_comp, self.s_out):
            s.wait_stream(cur)
        ev = lambda: torch.cuda.Event()
        in_ready, comp_done, grad_out = [ev(), ev()], [ev(), ev()], [ev(), ev()]
        img_out = None
        for i in range(len(host_in)):
            s = i & 1
            d_in, d_grad = self.d_in[s], self.d_grad[s]
            if i >= 2:
                self.s_in.wait_event(comp_done[s])  # step i-2 no longer reads this slot
            with torch.cuda.stream(self.s_in):
                d_in.copy_(host_in[i], non_blocking=True)
                in_ready[s].record(self.s_in)
            self.s_comp.wait_event(in_ready[s])
            if img_out is not None:
                self.s_comp.wait_event(img_out)  # the image buffer has been read out
            with torch.cuda.stream(self.s_comp):
                if self.graphs is not None:
                    self.graphs[s][0].replay()
                else:
                    self._fwd(s)
            img_ready = ev()
            img_ready.record(self.s_comp)
            if i >= 2:
                self.s_comp.wait_event(grad_out[s])  # step i-2's gradients have left this slot
            with torch.cuda.stream(self.s_comp):
                if self.graphs is not None:
                    self.graphs[s][1].replay()
                else:
                    self._bwd(s)
            comp_done[s].record(self.s_comp)
            with torch.cuda.stream(self.s_out):
                self.s_out.wait_event(img_ready)
                host_img[i].copy_(rast.rgba, non_blocking=True)
                img_out = ev()
                img_out.record(self.s_out)
                self.s_out.wait_event(comp_done[s])
                host_grad[i].copy_(d_grad, non_blocking=True)
                grad_out[s].record(self.s_out)
        for s in (self.s_in, self.s_comp, self.s_out):
            cur.wait_stream(s)

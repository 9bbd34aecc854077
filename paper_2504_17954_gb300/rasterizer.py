"""PyTorch-facing wrapper of libivrgs: device buffers, streams and a torch.autograd.Function.

PyTorch provides device memory and the current stream; every computation runs in the
library's kernels (``_native``). Nothing here computes any part of the rendering.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import List, Optional, Sequence

import torch

from . import _native as N

ATTRS = ("mean", "log_scale", "quat", "opacity_logit", "dcolor", "normal", "kads")
WIDTH = {"mean": 3, "log_scale": 3, "quat": 4, "opacity_logit": 1, "dcolor": 3, "normal": 3, "kads": 4}


def _vp(t: Optional[torch.Tensor]):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _stream(stream=None) -> C.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _check_cuda(t: torch.Tensor, name: str, dtype=torch.float32):
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")


# ----------------------------------------------------------------------------------------
@dataclass
class Gaussians:
    """Editable Gaussians on the device, structure of arrays (Sec. 4.3 attribute set).

    precision 0 (float32), 1 (16-bit storage, see ``pack_mixed``) or 2 (vector-quantised, see
    ``vq_compress``); ``anchor`` holds the float32 position anchors of the 16-bit storage,
    ``codebook`` / ``vq_k`` the per-model codebooks of the quantised storage."""
    mean: torch.Tensor
    log_scale: torch.Tensor
    quat: torch.Tensor
    opacity_logit: torch.Tensor
    dcolor: torch.Tensor
    normal: torch.Tensor
    kads: torch.Tensor
    model_id: Optional[torch.Tensor]
    n_models: int
    precision: int = 0
    anchor: Optional[torch.Tensor] = None
    codebook: Optional[torch.Tensor] = None
    vq_k: int = 0
    sh: Optional[torch.Tensor] = None  # [n, (sh_degree + 1)^2, 3] float32: 3DGS colour instead of Blinn-Phong
    sh_degree: int = -1

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    def struct(self, tensors: Optional[Sequence[torch.Tensor]] = None) -> N.ivrgs_gaussians:
        ts = [getattr(self, k) for k in ATTRS] if tensors is None else list(tensors)
        s = N.ivrgs_gaussians()
        s.n = self.n
        s.precision = self.precision
        s.n_models = self.n_models
        for k, t in zip(ATTRS, ts):
            setattr(s, k, t.data_ptr())
        s.model_id = self.model_id.data_ptr() if self.model_id is not None else None
        s.anchor = self.anchor.data_ptr() if self.anchor is not None else None
        s.codebook = self.codebook.data_ptr() if self.codebook is not None else None
        s.vq_k = int(self.vq_k)
        s.sh = self.sh.data_ptr() if self.sh is not None else None
        s.sh_degree = int(self.sh_degree)
        return s

    @staticmethod
    def empty(n: int, n_models: int, device="cuda") -> "Gaussians":
        z = lambda w: torch.empty((n, w) if w > 1 else (n,), dtype=torch.float32, device=device)
        return Gaussians(*(z(WIDTH[k]) for k in ATTRS), model_id=torch.empty(n, dtype=torch.int16, device=device),
                         n_models=n_models)

    @staticmethod
    def empty_mixed(n: int, n_models: int, device="cuda") -> "Gaussians":
        h = lambda w, dt: torch.empty((n, w) if w > 1 else (n,), dtype=dt, device=device)
        n_chunks = (n + N.IVRGS_ANCHOR_CHUNK - 1) // N.IVRGS_ANCHOR_CHUNK
        return Gaussians(mean=h(3, torch.float16), log_scale=h(3, torch.bfloat16), quat=h(4, torch.float16),
                         opacity_logit=h(1, torch.float16), dcolor=h(3, torch.bfloat16), normal=h(3, torch.bfloat16),
                         kads=h(4, torch.float16), model_id=torch.empty(n, dtype=torch.int16, device=device),
                         n_models=n_models, precision=N.IVRGS_MIXED,
                         anchor=torch.empty((max(n_chunks, 1), 3), dtype=torch.float32, device=device))

    @staticmethod
    def from_arrays(arrs: dict, n_models: int = 1, device="cuda") -> "Gaussians":
        t = lambda a: torch.as_tensor(a, dtype=torch.float32).to(device).contiguous()
        return Gaussians(*(t(arrs[k]) for k in ATTRS), model_id=None, n_models=n_models)


def vq_compress(g: Gaussians, k: int = 256, iters: int = 16, stream=None) -> Gaussians:
    """Vector-quantised storage of float32 Gaussians (Sec. 4.4; ivrgs_vq_build): per basic
    model and attribute (all but mean and normal) a k-entry scalar codebook from ``iters``
    Lloyd (k-means) iterations on the device, and one uint8 index per component. Mean, normal
    and model ids are shared with ``g``."""
    if g.precision != N.IVRGS_FP32 or g.model_id is None:
        raise ValueError("vq_compress takes float32 Gaussians with model ids")
    dev = g.mean.device
    u8 = lambda w: torch.empty((g.n, w) if w > 1 else (g.n,), dtype=torch.uint8, device=dev)
    out = Gaussians(mean=g.mean, log_scale=u8(3), quat=u8(4), opacity_logit=u8(1), dcolor=u8(3), normal=g.normal,
                    kads=u8(4), model_id=g.model_id, n_models=g.n_models, precision=N.IVRGS_VQ,
                    codebook=torch.empty((g.n_models, N.IVRGS_VQ_ATTRS, k), dtype=torch.float32, device=dev),
                    vq_k=k)
    gs, os_ = g.struct(), out.struct()
    wsb = N.ivrgs_vq_build_workspace(g.n_models, k)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    N.ivrgs_vq_build(C.byref(gs), k, iters, C.byref(os_), _vp(ws), wsb, _stream(stream))
    return out


def pack_mixed(g: Gaussians, lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0), stream=None):
    """16-bit storage of float32 Gaussians (ivrgs_morton_keys + ivrgs_pack_mixed).

    The Gaussians are reordered by (model, Morton code inside the box [lo, hi]) so that every
    chunk of 256 is spatially compact; the permutation (a one-time model preparation, sorted
    with torch) is returned with the packed set: packed[k] = g[order[k]]."""
    if g.precision != N.IVRGS_FP32:
        raise ValueError("pack_mixed takes float32 Gaussians")
    dev = g.mean.device
    keys = torch.empty(g.n, dtype=torch.int64, device=dev)
    lo_c, hi_c = (C.c_float * 3)(*lo), (C.c_float * 3)(*hi)
    gs = g.struct()
    N.ivrgs_morton_keys(C.byref(gs), lo_c, hi_c, _vp(keys), _stream(stream))
    order = torch.argsort(keys, stable=True).to(torch.int32)
    out = Gaussians.empty_mixed(g.n, g.n_models, dev)
    os_ = out.struct()
    N.ivrgs_pack_mixed(C.byref(gs), _vp(order), C.byref(os_), _stream(stream))
    return out, order


def reorder_spatial(g: Gaussians, lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0), stream=None):
    """Float32 Gaussians reordered by (model, Morton code inside the box [lo, hi]), the order
    pack_mixed gives its chunks: a one-time layout step of a composed set (the permutation is
    sorted with torch and applied by gathers). Gaussians close in space are then close in
    memory, so the binning's depth-ordered gathers and the compositing's per-tile gathers touch
    fewer DRAM lines. Images and gradients are unchanged, except that exactly equal depths
    composite in the new composed order. Returns (reordered, order), reordered[k] = g[order[k]]."""
    if g.precision != N.IVRGS_FP32:
        raise ValueError("reorder_spatial takes float32 Gaussians")
    dev = g.mean.device
    keys = torch.empty(g.n, dtype=torch.int64, device=dev)
    lo_c, hi_c = (C.c_float * 3)(*lo), (C.c_float * 3)(*hi)
    gs = g.struct()
    N.ivrgs_morton_keys(C.byref(gs), lo_c, hi_c, _vp(keys), _stream(stream))
    order = torch.argsort(keys, stable=True)
    take = lambda t: t.index_select(0, order).contiguous() if t is not None else None
    out = Gaussians(*(take(getattr(g, k)) for k in ATTRS), model_id=take(g.model_id), n_models=g.n_models,
                    sh=take(g.sh), sh_degree=g.sh_degree)
    return out, order.to(torch.int32)


def edit_structs(palette, opacity_scale, visible, lam, bias, light_dir=None):
    M = len(opacity_scale)
    ed = (N.ivrgs_model_edit * M)()
    for m in range(M):
        for k in range(3):
            ed[m].palette[k] = float(palette[m][k])
        ed[m].opacity_scale = float(opacity_scale[m])
        ed[m].visible = int(bool(visible[m]))
    li = N.ivrgs_light()
    for k in range(4):
        li.lambda_[k] = float(lam[k])
        li.bias[k] = float(bias[k])
    if light_dir is not None:
        for k in range(3):
            li.dir[k] = float(light_dir[k])
        li.dir_on = 1
    return ed, li


def compose_edit(models: Sequence[Gaussians], palette, opacity_scale, visible, lam, bias, device="cuda",
                 composed: Optional[Gaussians] = None, edit_table: Optional[torch.Tensor] = None, stream=None,
                 light_dir=None):
    """Concatenate basic models on the device and write the edit table (ivrgs_compose_edit).

    With ``models`` empty (or None) and ``composed`` None only the edit table is rewritten.
    ``light_dir`` (3 floats) switches on the global light that replaces every orbital view's."""
    M = len(opacity_scale)
    ed, li = edit_structs(palette, opacity_scale, visible, lam, bias, light_dir)
    if edit_table is None:
        edit_table = torch.empty(N.lib().ivrgs_edit_table_floats(M), dtype=torch.float32, device=device)
    comp_s = None
    arr = None
    if models:
        n = sum(m.n for m in models)
        if composed is None:
            composed = Gaussians.empty(n, M, device)
        arr = (N.ivrgs_gaussians * M)(*[m.struct() for m in models])
        comp_s = composed.struct()
    N.ivrgs_compose_edit(arr, M, ed, C.byref(li), C.byref(comp_s) if comp_s is not None else None,
                         _vp(edit_table), _stream(stream))
    return composed, edit_table


# ----------------------------------------------------------------------------------------
def camera_structs(cams) -> (C.Array, int):
    """Pack cameras (objects with W, H, fx, fy, cx, cy, R, t, campos, znear, headlight, light_dir)."""
    V = len(cams)
    arr = (N.ivrgs_camera * V)()
    off = 0
    for v, c in enumerate(cams):
        a = arr[v]
        a.W, a.H = int(c.W), int(c.H)
        a.fx, a.fy, a.cx, a.cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
        for k in range(9):
            a.R[k] = float(c.R[k])
        for k in range(3):
            a.t[k] = float(c.t[k])
            a.campos[k] = float(c.campos[k])
            a.light_dir[k] = float(c.light_dir[k])
        a.znear = float(c.znear)
        a.headlight = int(c.headlight)
        a.pix_offset = off
        off += int(c.W) * int(c.H)
    return arr, off


def n_tiles(cams, tile_w: int = 16, tile_h: int = 16) -> int:
    return sum(((c.W + tile_w - 1) // tile_w) * ((c.H + tile_h - 1) // tile_h) for c in cams)


class Rasterizer:
    """Device buffers for one camera set and one scene size; forward and backward calls.

    ``capacity`` fixes the pair buffer (required for CUDA-graph capture, mode="capacity");
    with mode="exact" the buffer grows to the exact pair count when needed. ``cull`` drops the
    pairs of tiles that the Gaussian's opacity cut-off ellipse misses (IVRGS_BIN_CULL): the same
    images and gradients from shorter tile lists; ``cull=False`` gives the full rectangle lists.

    ``tile_h`` is the tile height (16 or 8; tiles are 16 pixels wide): a launch shape, which
    the autotuner's ``tune_tiles`` can pick per workload.

    ``generation`` counts the eager calls that rewrite the per-render state (projection,
    binning, compositing); ``RenderFunction`` uses it to refuse a backward whose forward state
    has since been overwritten. Replays of a captured graph do not advance it.
    """

    def __init__(self, cams, n_gaussians: int, n_models: int, device="cuda", capacity: Optional[int] = None,
                 lowpass: float = 0.3, bg=(0.0, 0.0, 0.0), cull: bool = True, tile_h: int = 16):
        self.cams = list(cams)
        self.V = len(self.cams)
        self.n = int(n_gaussians)
        self.n_models = int(n_models)
        self.device = torch.device(device)
        self.lowpass = float(lowpass)
        self.cull_flag = N.IVRGS_BIN_CULL if cull else 0
        self.cam_arr, self.n_pix = camera_structs(self.cams)
        self.bg = (C.c_float * 3)(*[float(x) for x in bg])
        if tile_h not in (16, 8):
            raise ValueError("tile_h must be 16 or 8")
        self.tile_h = int(tile_h)
        self.n_tiles = n_tiles(self.cams, 16, self.tile_h)
        VN = self.V * self.n
        dev = self.device
        self.xy = torch.empty((VN, 2), dtype=torch.float32, device=dev)
        self.conic_o = torch.empty((VN, 4), dtype=torch.float32, device=dev)
        self.rgbd = torch.empty((VN, 4), dtype=torch.float32, device=dev)
        self.radius = torch.empty(VN, dtype=torch.int32, device=dev)
        self.rgba = torch.empty((self.n_pix, 4), dtype=torch.float32, device=dev)
        self.final_T = torch.empty(self.n_pix, dtype=torch.float32, device=dev)
        self.last = torch.empty(self.n_pix, dtype=torch.int32, device=dev)
        self.ranges = torch.empty((self.n_tiles, 2), dtype=torch.int32, device=dev)
        self.d_n_pairs = torch.zeros(1, dtype=torch.int64, device=dev)
        self.n_pairs = 0
        self.tiles = self.values = self.ws_bin = None
        self.capacity = 0
        self._ensure_capacity(int(capacity) if capacity else max(1024, 8 * VN))
        self.ws_bwd_bytes = N.ivrgs_render_backward_workspace(self.n, self.V)
        self.ws_bwd = None
        self.edit_grad = torch.empty(N.lib().ivrgs_edit_table_floats(self.n_models) + 4 * self.V,
                                     dtype=torch.float32, device=dev)
        self.generation = 0

    # -- buffers
    def _ensure_capacity(self, cap: int):
        cap = min(int(cap), N.IVRGS_MAX_PAIRS - 1)
        if cap <= self.capacity:
            return
        self.capacity = cap
        self.tiles = torch.empty(cap, dtype=torch.int32, device=self.device)
        self.values = torch.empty(cap, dtype=torch.int32, device=self.device)
        self.ws_bin_bytes = N.ivrgs_bin_workspace(self.n, self.V, self.cam_arr, 16, self.tile_h, cap)
        self.ws_bin = torch.empty(self.ws_bin_bytes, dtype=torch.uint8, device=self.device)

    def projected_struct(self) -> N.ivrgs_projected:
        p = N.ivrgs_projected()
        p.n, p.n_views = self.n, self.V
        p.xy, p.conic_o, p.rgbd, p.radius = (t.data_ptr() for t in (self.xy, self.conic_o, self.rgbd, self.radius))
        return p

    def bins_struct(self) -> N.ivrgs_bins:
        b = N.ivrgs_bins()
        b.tile_w, b.tile_h = 16, self.tile_h
        b.n_tiles = self.n_tiles
        b.capacity = self.capacity
        b.tiles, b.values = self.tiles.data_ptr(), self.values.data_ptr()
        b.ranges = self.ranges.data_ptr()
        b.d_n_pairs = self.d_n_pairs.data_ptr()
        b.n_pairs = self.n_pairs
        return b

    # -- steps
    def project(self, g: Gaussians, edit_table: torch.Tensor, stream=None, tensors=None):
        self.generation += 1
        gs = g.struct(tensors)
        p = self.projected_struct()
        N.ivrgs_project(C.byref(gs), _vp(edit_table), self.cam_arr, self.V, self.lowpass, C.byref(p), _stream(stream))

    def bin(self, mode: str = "exact", stream=None) -> int:
        self.generation += 1
        p = self.projected_struct()
        if mode == "exact":
            while True:
                b = self.bins_struct()
                st = N.ivrgs_bin(C.byref(p), self.cam_arr, self.V, N.IVRGS_BIN_EXACT | self.cull_flag, _vp(self.ws_bin),
                                 self.ws_bin_bytes, C.byref(b), _stream(stream),
                                 allow=(N.IVRGS_OK, N.IVRGS_ERR_CAPACITY))
                if st == N.IVRGS_OK:
                    self.n_pairs = int(b.n_pairs)
                    return self.n_pairs
                need = int(b.n_pairs)
                if need >= N.IVRGS_MAX_PAIRS:
                    raise N.IvrgsError("ivrgs_bin", st, f"{need} pairs exceed the per-call limit")
                self._ensure_capacity(int(need * 1.25) + 1024)
        b = self.bins_struct()
        N.ivrgs_bin(C.byref(p), self.cam_arr, self.V, N.IVRGS_BIN_CAPACITY | self.cull_flag, _vp(self.ws_bin),
                    self.ws_bin_bytes, C.byref(b), _stream(stream))
        return -1

    def render(self, stream=None):
        self.generation += 1
        p, b = self.projected_struct(), self.bins_struct()
        N.ivrgs_render(C.byref(p), C.byref(b), self.cam_arr, self.V, self.bg, _vp(self.rgba), _vp(self.final_T),
                       _vp(self.last), _stream(stream))
        return self.rgba

    def forward(self, g: Gaussians, edit_table: torch.Tensor, mode: str = "exact", stream=None, tensors=None):
        self.project(g, edit_table, stream, tensors)
        self.bin(mode, stream)
        return self.render(stream)

    AUX_CHANNELS = ("depth", "nx", "ny", "nz", "dc_r", "dc_g", "dc_b", "ka", "kd", "ks", "beta", "alpha")

    def render_aux(self, g: Gaussians, edit_table: torch.Tensor, stream=None) -> torch.Tensor:
        """Auxiliary maps of the last forward (ivrgs_render_aux): [n_pix, 12] with the channels
        AUX_CHANNELS (depth, normal, offset colour, k', 1 - T)."""
        if getattr(self, "aux", None) is None:
            self.aux = torch.empty((self.n_pix, 12), dtype=torch.float32, device=self.device)
        gs = g.struct()
        p, b = self.projected_struct(), self.bins_struct()
        N.ivrgs_render_aux(C.byref(gs), _vp(edit_table), C.byref(p), C.byref(b), self.cam_arr, self.V,
                           _vp(self.aux), _stream(stream))
        return self.aux

    def render_aux_backward(self, g: Gaussians, edit_table: torch.Tensor, dL_daux: torch.Tensor,
                            grad: Optional[Gaussians] = None, stream=None):
        """Reverse mode of render_aux for the last forward (ivrgs_render_aux_backward): dL_daux
        [n_pix, 12] over the channels of render_aux. Returns (grad, gradient of the edit table)."""
        _check_cuda(dL_daux, "dL_daux")
        if getattr(self, "ws_aux_bwd", None) is None:
            self.ws_aux_bwd_bytes = N.ivrgs_render_aux_backward_workspace(self.n, self.V)
            self.ws_aux_bwd = torch.empty(self.ws_aux_bwd_bytes, dtype=torch.uint8, device=self.device)
        if grad is None:
            grad = Gaussians.empty(self.n, self.n_models, self.device)
            grad.model_id = None
        if g.sh is not None and grad.sh is None:
            grad.sh = torch.empty_like(g.sh)
            grad.sh_degree = g.sh_degree
        gs, gr = g.struct(), grad.struct()
        p, b = self.projected_struct(), self.bins_struct()
        eg = torch.empty_like(self.edit_grad)
        N.ivrgs_render_aux_backward(C.byref(gs), _vp(edit_table), C.byref(p), C.byref(b), self.cam_arr, self.V,
                                    self.lowpass, _vp(self.final_T), _vp(self.last), _vp(dL_daux), _vp(self.ws_aux_bwd),
                                    self.ws_aux_bwd_bytes, C.byref(gr), _vp(eg), _stream(stream))
        return grad, eg

    def backward(self, g: Gaussians, edit_table: torch.Tensor, dL_drgba: torch.Tensor, grad: Optional[Gaussians] = None,
                 stream=None, tensors=None, accumulate: bool = False, edit_grad: Optional[torch.Tensor] = None):
        _check_cuda(dL_drgba, "dL_drgba")
        if self.ws_bwd is None:
            self.ws_bwd = torch.empty(self.ws_bwd_bytes, dtype=torch.uint8, device=self.device)
        if grad is None:
            grad = Gaussians.empty(self.n, self.n_models, self.device)
            grad.model_id = None
        if g.sh is not None and grad.sh is None:
            grad.sh = torch.empty_like(g.sh)
            grad.sh_degree = g.sh_degree
        gs = g.struct(tensors)
        gr = grad.struct()
        p, b = self.projected_struct(), self.bins_struct()
        eg = self.edit_grad if edit_grad is None else edit_grad
        fn = N.ivrgs_render_backward_accumulate if accumulate else N.ivrgs_render_backward
        fn(C.byref(gs), _vp(edit_table), C.byref(p), C.byref(b), self.cam_arr, self.V, self.lowpass, self.bg,
           _vp(self.final_T), _vp(self.last), _vp(dL_drgba), _vp(self.ws_bwd), self.ws_bwd_bytes, C.byref(gr),
           _vp(eg), _stream(stream))
        return grad, eg

    # -- CUDA graphs
    def capture(self, g: Gaussians, edit_table: torch.Tensor, dL_drgba: Optional[torch.Tensor] = None,
                grad: Optional[Gaussians] = None, warmup: int = 2, loss=None) -> "torch.cuda.CUDAGraph":
        """Capture one step (projection, CAPACITY-mode binning, compositing and, if dL_drgba is
        given, the backward into ``grad``) as a CUDA graph; ``graph.replay()`` reruns it on the
        current contents of the Gaussian, edit-table and dL buffers. ``loss``, if given, is called
        (and captured) between the compositing and the backward, e.g. an image loss that writes
        dL_drgba from ``self.rgba``.

        The pair buffer must already hold the step's pairs (run ``forward(mode="exact")`` once);
        after a replay, ``d_n_pairs > capacity`` means the step overflowed and must be rerun
        with a larger capacity."""
        if dL_drgba is not None:
            _check_cuda(dL_drgba, "dL_drgba")
            if self.ws_bwd is None:
                self.ws_bwd = torch.empty(self.ws_bwd_bytes, dtype=torch.uint8, device=self.device)
            if grad is None:
                grad = Gaussians.empty(self.n, self.n_models, self.device)
                grad.model_id = None
        self.graph_grad = grad
        N.prof_enable(False)
        side = torch.cuda.Stream(device=self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        def step():
            self.forward(g, edit_table, mode="capacity")
            if loss is not None:
                loss()
            if dL_drgba is not None:
                self.backward(g, edit_table, dL_drgba, grad=grad)

        with torch.cuda.stream(side):  # warm-up outside capture (lazy module loading etc.)
            for _ in range(warmup):
                step()
        torch.cuda.current_stream(self.device).wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        return graph

    # -- views of the packed image
    def view_image(self, v: int, t: Optional[torch.Tensor] = None) -> torch.Tensor:
        t = self.rgba if t is None else t
        c = self.cams[v]
        off = self.cam_arr[v].pix_offset
        return t[off:off + c.W * c.H].view(c.H, c.W, *t.shape[1:])


# ----------------------------------------------------------------------------------------
def plan_waves(cams, n_gaussians: int, max_views: int = 32, pixel_budget: int = 24 << 20, tile_h: int = 16,
               max_tiles: int = 1 << 16) -> List[List[int]]:
    """Consecutive groups of view indices, in view order, each rendered by one set of calls:
    at most ``max_views`` views, and fewer than the library's 2^30 records (n_gaussians * views)
    per binning call; a wave closes before a view that would take its pixels over
    ``pixel_budget`` or its tiles (16 x tile_h) over ``max_tiles`` (a single view larger than
    either forms a wave of its own). With at most 2^16 tiles per call the tile ids travel through
    the radix sort as 16-bit keys in two passes instead of three."""
    max_views = max(1, min(max_views, (N.IVRGS_MAX_PAIRS - 1) // max(n_gaussians, 1)))
    waves: List[List[int]] = []
    cur, pix, tiles = [], 0, 0
    for v, c in enumerate(cams):
        t = n_tiles([c], 16, tile_h)
        if cur and (len(cur) >= max_views or pix + c.W * c.H > pixel_budget or tiles + t > max_tiles):
            waves.append(cur)
            cur, pix, tiles = [], 0, 0
        cur.append(v)
        pix += c.W * c.H
        tiles += t
    if cur:
        waves.append(cur)
    return waves


class WaveRasterizer:
    """Many views rendered in waves of at most ``max_views`` views and ``pixel_budget`` pixels
    (so that no binning call exceeds the library's per-call pair limit); the backward sums the
    waves' gradients with ivrgs_render_backward_accumulate. Each wave owns a Rasterizer."""

    def __init__(self, cams, n_gaussians: int, n_models: int, device="cuda", lowpass: float = 0.3,
                 bg=(0.0, 0.0, 0.0), max_views: int = 32, pixel_budget: int = 24 << 20, cull: bool = True,
                 tile_h: int = 16):
        self.cams = list(cams)
        self.waves: List[List[int]] = plan_waves(self.cams, n_gaussians, max_views, pixel_budget, tile_h)
        self.rasts = [Rasterizer([self.cams[v] for v in wv], n_gaussians, n_models, device=device, lowpass=lowpass,
                                 bg=bg, cull=cull, tile_h=tile_h) for wv in self.waves]
        self.n_models = n_models
        self.V = len(self.cams)

    def forward(self, g: Gaussians, edit_table: torch.Tensor, mode: str = "exact"):
        for r in self.rasts:
            r.forward(g, edit_table, mode=mode)

    def backward(self, g: Gaussians, edit_table: torch.Tensor, dL_per_wave: Sequence[torch.Tensor],
                 grad: Optional[Gaussians] = None):
        """dL_per_wave[k]: packed dL/dRGBA of wave k's views. Returns (grad, gradient of the
        edit table, per-view light gradients [V, 3]); the waves' contributions are summed."""
        ne = edit_table.numel()
        dev = self.rasts[0].device
        eg = torch.empty(ne + 4 * max(len(wv) for wv in self.waves), dtype=torch.float32, device=dev)
        light = torch.zeros((self.V, 3), dtype=torch.float32, device=dev)
        for k, (r, wv) in enumerate(zip(self.rasts, self.waves)):
            grad, _ = r.backward(g, edit_table, dL_per_wave[k], grad=grad, accumulate=k > 0, edit_grad=eg)
            light[wv] = eg[ne:ne + 4 * len(wv)].view(len(wv), 4)[:, :3]
        return grad, eg[:ne], light

    def view_image(self, v: int) -> torch.Tensor:
        for r, wv in zip(self.rasts, self.waves):
            if v in wv:
                return r.view_image(wv.index(v))
        raise IndexError(v)

    def size_buffers(self, g: Gaussians, edit_table: torch.Tensor, slack: float = 1.1):
        """One EXACT-mode forward per wave, then pair buffers with ``slack`` times the counts:
        what CAPACITY-mode binning (and so ``capture``) needs."""
        for r in self.rasts:
            r.forward(g, edit_table, mode="exact")
        torch.cuda.synchronize()
        for r in self.rasts:
            r._ensure_capacity(int(r.n_pairs * slack) + 4096)

    def overflowed(self) -> bool:
        """True if a wave's last CAPACITY-mode binning had more pairs than its buffer holds."""
        return any(int(r.d_n_pairs.item()) > r.capacity for r in self.rasts)

    def capture(self, g: Gaussians, edit_table: torch.Tensor, dL_per_wave: Optional[Sequence[torch.Tensor]] = None,
                grad: Optional[Gaussians] = None, warmup: int = 2) -> "torch.cuda.CUDAGraph":
        """Every wave's projection, CAPACITY-mode binning and compositing and, with
        ``dL_per_wave``, the backward summed over the waves (into ``grad``, ``self.edit_grad`` and
        ``self.light_grad``) as ONE CUDA graph; ``graph.replay()`` reruns the whole step on the
        current contents of the Gaussian, edit-table and dL buffers. Run ``size_buffers`` first;
        after a replay, ``overflowed()`` tells whether a wave must be re-sized and captured again."""
        dev = self.rasts[0].device
        ne = edit_table.numel()
        if dL_per_wave is not None and grad is None:
            grad = Gaussians.empty(self.rasts[0].n, self.n_models, dev)
            grad.model_id = None
        self.graph_grad = grad
        self.edit_grad = torch.zeros(ne + 4 * max(len(wv) for wv in self.waves), dtype=torch.float32, device=dev)
        self.light_grad = torch.zeros((self.V, 3), dtype=torch.float32, device=dev)
        # a graph writes through the raw addresses of these buffers: keep every captured graph's alive
        self._graph_buffers = getattr(self, "_graph_buffers", []) + [(grad, self.edit_grad, self.light_grad)]
        N.prof_enable(False)

        def step():
            for r in self.rasts:
                r.forward(g, edit_table, mode="capacity")
            if dL_per_wave is not None:
                for k, (r, wv) in enumerate(zip(self.rasts, self.waves)):
                    r.backward(g, edit_table, dL_per_wave[k], grad=grad, accumulate=k > 0, edit_grad=self.edit_grad)
                    self.light_grad[wv[0]:wv[-1] + 1] = self.edit_grad[ne:ne + 4 * len(wv)].view(len(wv), 4)[:, :3]

        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            for _ in range(warmup):
                step()
        torch.cuda.current_stream(dev).wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        return graph


# ----------------------------------------------------------------------------------------
class RenderFunction(torch.autograd.Function):
    """rgba = render(Gaussian attributes, edit table); backward through ivrgs_render_backward.

    The forward keeps only the projected records, the bins, the final transmittance and the
    last-contributor index per pixel (inside the Rasterizer); the per-pixel transmittance
    of every contributor is recomputed in the backward, not stored. Because that state lives in
    the Rasterizer, a render's backward must run before the same Rasterizer renders again: a
    later forward on it makes the earlier render's backward raise (one Rasterizer per render
    that takes part in a loss). The per-view light-direction gradients of the last backward
    are left in ``rast.light_grad`` ([V, 3]).
    """

    @staticmethod
    def forward(ctx, rast: Rasterizer, g: Gaussians, edit_table, *attrs):
        rast.forward(g, edit_table.detach(), tensors=[a.detach() for a in attrs])
        ctx.rast, ctx.g = rast, g
        ctx.generation = rast.generation
        ctx.save_for_backward(edit_table, *attrs)
        return rast.rgba.clone()

    @staticmethod
    def backward(ctx, d_rgba):
        edit_table, *attrs = ctx.saved_tensors
        rast: Rasterizer = ctx.rast
        if rast.generation != ctx.generation:
            raise RuntimeError("render(): the Rasterizer has rendered again since this forward, so the "
                               "records, tile lists and per-pixel state its backward needs are gone; "
                               "use one Rasterizer per render that takes part in a loss")
        grad, egrad = rast.backward(ctx.g, edit_table.detach(), d_rgba.contiguous(),
                                    tensors=[a.detach() for a in attrs])
        ne = edit_table.numel()
        rast.light_grad = egrad[ne:].view(rast.V, 4)[:, :3].clone()
        outs = [getattr(grad, k).view_as(a) for k, a in zip(ATTRS, attrs)]
        return (None, None, egrad[:ne].clone(), *outs)


def render(rast: Rasterizer, g: Gaussians, edit_table: torch.Tensor, params: Optional[Sequence[torch.Tensor]] = None):
    """Differentiable render of all views; returns the packed [n_pix, 4] RGBA tensor."""
    attrs = [getattr(g, k) for k in ATTRS] if params is None else list(params)
    return RenderFunction.apply(rast, g, edit_table, *attrs)

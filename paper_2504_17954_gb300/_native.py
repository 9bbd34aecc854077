"""ctypes binding of libivrgs.so: the C-ABI structs and entry points under their C names.

Argument marshalling only. Every step of the path runs in the library's CUDA kernels; if the
library is missing or fails to load this module raises, there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libivrgs.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "ivrgs.h")

IVRGS_OK = 0
IVRGS_ERR_INVALID_ARG = 1
IVRGS_ERR_CAPACITY = 2
IVRGS_ERR_CUDA = 3
IVRGS_ERR_TIMEOUT = 4
IVRGS_ERR_UNSUPPORTED = 5
IVRGS_MAX_VIEWS = 128
IVRGS_MAX_MODELS = 1024
IVRGS_EDIT_STRIDE = 8
IVRGS_MAX_PAIRS = 1 << 30
IVRGS_FP32 = 0
IVRGS_MIXED = 1
IVRGS_VQ = 2
IVRGS_VQ_ATTRS = 8
IVRGS_VQ_MAX_K = 256
IVRGS_ANCHOR_CHUNK = 256
IVRGS_BIN_EXACT = 0
IVRGS_BIN_CAPACITY = 1
IVRGS_BIN_CULL = 2
IVRGS_LEARN_COLOR = 1
IVRGS_LEARN_OPACITY = 2
IVRGS_LEARN_LIGHT_MAGNITUDE = 4
IVRGS_LEARN_LIGHT_DIRECTION = 8

STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CAPACITY", 3: "CUDA_ERROR", 4: "TIMEOUT", 5: "UNSUPPORTED"}


class ivrgs_camera(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("R", C.c_float * 9), ("t", C.c_float * 3), ("campos", C.c_float * 3),
                ("znear", C.c_float), ("headlight", C.c_int32), ("light_dir", C.c_float * 3),
                ("pix_offset", C.c_int64)]


class ivrgs_model_edit(C.Structure):
    _fields_ = [("palette", C.c_float * 3), ("opacity_scale", C.c_float), ("visible", C.c_int32)]


class ivrgs_light(C.Structure):
    _fields_ = [("lambda_", C.c_float * 4), ("bias", C.c_float * 4), ("dir", C.c_float * 3), ("dir_on", C.c_int32)]


class ivrgs_gaussians(C.Structure):
    _fields_ = [("n", C.c_int64), ("precision", C.c_int32), ("n_models", C.c_int32), ("mean", C.c_void_p),
                ("log_scale", C.c_void_p), ("quat", C.c_void_p), ("opacity_logit", C.c_void_p),
                ("dcolor", C.c_void_p), ("normal", C.c_void_p), ("kads", C.c_void_p), ("model_id", C.c_void_p),
                ("anchor", C.c_void_p), ("codebook", C.c_void_p), ("vq_k", C.c_int32), ("sh", C.c_void_p),
                ("sh_degree", C.c_int32)]


class ivrgs_projected(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_views", C.c_int32), ("xy", C.c_void_p), ("conic_o", C.c_void_p),
                ("rgbd", C.c_void_p), ("radius", C.c_void_p)]


class ivrgs_bins(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("n_tiles", C.c_int64), ("capacity", C.c_int64),
                ("tiles", C.c_void_p), ("values", C.c_void_p), ("ranges", C.c_void_p), ("d_n_pairs", C.c_void_p),
                ("n_pairs", C.c_int64)]


_P = C.POINTER
_SIGNATURES = {
    "ivrgs_last_error": (C.c_char_p, []),
    "ivrgs_version": (C.c_int32, []),
    "ivrgs_set_option": (C.c_int32, [C.c_char_p, C.c_int64]),
    "ivrgs_get_option": (C.c_int32, [C.c_char_p, _P(C.c_int64)]),
    "ivrgs_edit_table_floats": (C.c_int64, [C.c_int32]),
    "ivrgs_compose_edit": (C.c_int32, [_P(ivrgs_gaussians), C.c_int32, _P(ivrgs_model_edit), _P(ivrgs_light),
                                       _P(ivrgs_gaussians), C.c_void_p, C.c_void_p]),
    "ivrgs_project": (C.c_int32, [_P(ivrgs_gaussians), C.c_void_p, _P(ivrgs_camera), C.c_int32, C.c_float,
                                  _P(ivrgs_projected), C.c_void_p]),
    "ivrgs_morton_keys": (C.c_int32, [_P(ivrgs_gaussians), _P(C.c_float), _P(C.c_float), C.c_void_p, C.c_void_p]),
    "ivrgs_pack_mixed": (C.c_int32, [_P(ivrgs_gaussians), C.c_void_p, _P(ivrgs_gaussians), C.c_void_p]),
    "ivrgs_bin_workspace": (C.c_int32, [C.c_int64, C.c_int32, _P(ivrgs_camera), C.c_int32, C.c_int32, C.c_int64,
                                        _P(C.c_size_t)]),
    "ivrgs_bin": (C.c_int32, [_P(ivrgs_projected), _P(ivrgs_camera), C.c_int32, C.c_int32, C.c_void_p, C.c_size_t,
                              _P(ivrgs_bins), C.c_void_p]),
    "ivrgs_bin_check": (C.c_int32, [C.c_void_p, C.c_void_p]),
    "ivrgs_render": (C.c_int32, [_P(ivrgs_projected), _P(ivrgs_bins), _P(ivrgs_camera), C.c_int32,
                                 _P(C.c_float), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ivrgs_render_aux": (C.c_int32, [_P(ivrgs_gaussians), C.c_void_p, _P(ivrgs_projected), _P(ivrgs_bins),
                                     _P(ivrgs_camera), C.c_int32, C.c_void_p, C.c_void_p]),
    "ivrgs_render_aux_backward_workspace": (C.c_int32, [C.c_int64, C.c_int32, _P(C.c_size_t)]),
    "ivrgs_render_aux_backward": (C.c_int32, [_P(ivrgs_gaussians), C.c_void_p, _P(ivrgs_projected), _P(ivrgs_bins),
                                              _P(ivrgs_camera), C.c_int32, C.c_float, C.c_void_p, C.c_void_p,
                                              C.c_void_p, C.c_void_p, C.c_size_t, _P(ivrgs_gaussians), C.c_void_p,
                                              C.c_void_p]),
    "ivrgs_render_backward_workspace": (C.c_int32, [C.c_int64, C.c_int32, _P(C.c_size_t)]),
    "ivrgs_render_backward": (C.c_int32, [_P(ivrgs_gaussians), C.c_void_p, _P(ivrgs_projected), _P(ivrgs_bins),
                                          _P(ivrgs_camera), C.c_int32, C.c_float, _P(C.c_float), C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, _P(ivrgs_gaussians),
                                          C.c_void_p, C.c_void_p]),
    "ivrgs_render_backward_accumulate": (C.c_int32, [_P(ivrgs_gaussians), C.c_void_p, _P(ivrgs_projected),
                                                     _P(ivrgs_bins), _P(ivrgs_camera), C.c_int32, C.c_float,
                                                     _P(C.c_float), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                                     C.c_size_t, _P(ivrgs_gaussians), C.c_void_p, C.c_void_p]),
    "ivrgs_render_backward_static": (C.c_int32, [_P(ivrgs_gaussians), C.c_void_p, _P(ivrgs_projected),
                                                 _P(ivrgs_bins), _P(ivrgs_camera), C.c_int32, C.c_float,
                                                 _P(C.c_float), C.c_void_p, C.c_void_p, C.c_void_p,
                                                 _P(ivrgs_gaussians), C.c_void_p, C.c_void_p]),
    "ivrgs_image_loss_workspace": (C.c_int32, [_P(ivrgs_camera), C.c_int32, _P(C.c_size_t)]),
    "ivrgs_image_loss": (C.c_int32, [C.c_void_p, C.c_void_p, _P(ivrgs_camera), C.c_int32, C.c_float, C.c_void_p,
                                     C.c_size_t, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ivrgs_edit_adam_state_floats": (C.c_int64, [C.c_int32]),
    "ivrgs_edit_adam_init": (C.c_int32, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "ivrgs_edit_adam": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_float, C.c_float,
                                    C.c_float, C.c_float, C.c_void_p]),
    "ivrgs_vq_build_workspace": (C.c_int32, [C.c_int32, C.c_int32, _P(C.c_size_t)]),
    "ivrgs_vq_build": (C.c_int32, [_P(ivrgs_gaussians), C.c_int32, C.c_int32, _P(ivrgs_gaussians), C.c_void_p,
                                   C.c_size_t, C.c_void_p]),
    "ivrgs_debug_bin_hooks": (None, [C.c_longlong, C.c_longlong]),
    "ivrgs_prof_enable": (None, [C.c_int32]),
    "ivrgs_prof_report": (C.c_int64, [C.c_char_p, C.c_int64]),
}

_lib = None


class IvrgsError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__(f"{fn} failed: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib():
    """Load libivrgs.so (built in-tree by ``build.build()``); raises if it is absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libivrgs.so not built ({LIB_PATH}); run paper_2504_17954_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def declared_symbols():
    """Entry points declared in include/ivrgs.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ivrgs_[a-z_0-9]+)\s*\(", text)))


def last_error() -> str:
    return lib().ivrgs_last_error().decode()


def check(fn: str, status: int):
    if status != IVRGS_OK:
        raise IvrgsError(fn, status, last_error())


def call(fn: str, *args, allow=(IVRGS_OK,)):
    """Call an entry point; raise unless its status is in `allow`."""
    st = getattr(lib(), fn)(*args)
    if st not in allow:
        raise IvrgsError(fn, st, last_error())
    return st


# thin wrappers with the C names -------------------------------------------------------------
def ivrgs_compose_edit(models, n_models, edits, light, composed, d_edit_table, stream):
    return call("ivrgs_compose_edit", models, n_models, edits, light, composed, d_edit_table, stream)


def ivrgs_project(g, d_edit_table, cams, n_views, lowpass, out, stream):
    return call("ivrgs_project", g, d_edit_table, cams, n_views, lowpass, out, stream)


def ivrgs_morton_keys(g, lo, hi, d_keys, stream):
    return call("ivrgs_morton_keys", g, lo, hi, d_keys, stream)


def ivrgs_pack_mixed(g_in, d_order, g_out, stream):
    return call("ivrgs_pack_mixed", g_in, d_order, g_out, stream)


def ivrgs_bin_workspace(n, n_views, cams, tile_w, tile_h, capacity) -> int:
    b = C.c_size_t(0)
    call("ivrgs_bin_workspace", n, n_views, cams, tile_w, tile_h, capacity, C.byref(b))
    return int(b.value)


def ivrgs_bin(p, cams, n_views, mode, ws, ws_bytes, out, stream, allow=(IVRGS_OK,)):
    return call("ivrgs_bin", p, cams, n_views, mode, ws, ws_bytes, out, stream, allow=allow)


def ivrgs_bin_check(ws, stream, allow=(IVRGS_OK,)):
    return call("ivrgs_bin_check", ws, stream, allow=allow)


def ivrgs_render(p, b, cams, n_views, bg, d_rgba, d_final_T, d_last, stream):
    return call("ivrgs_render", p, b, cams, n_views, bg, d_rgba, d_final_T, d_last, stream)


def ivrgs_render_aux_backward_workspace(n, n_views) -> int:
    b = C.c_size_t(0)
    call("ivrgs_render_aux_backward_workspace", n, n_views, C.byref(b))
    return int(b.value)


def ivrgs_render_aux_backward(g, d_edit_table, p, b, cams, n_views, lowpass, d_final_T, d_last, d_dL, ws, ws_bytes,
                              grad, d_edit_grad, stream):
    return call("ivrgs_render_aux_backward", g, d_edit_table, p, b, cams, n_views, lowpass, d_final_T, d_last, d_dL,
                ws, ws_bytes, grad, d_edit_grad, stream)


def ivrgs_render_backward_workspace(n, n_views) -> int:
    b = C.c_size_t(0)
    call("ivrgs_render_backward_workspace", n, n_views, C.byref(b))
    return int(b.value)


def ivrgs_render_backward(g, d_edit_table, p, b, cams, n_views, lowpass, bg, d_final_T, d_last, d_dL, ws, ws_bytes,
                          grad, d_edit_grad, stream):
    return call("ivrgs_render_backward", g, d_edit_table, p, b, cams, n_views, lowpass, bg, d_final_T, d_last, d_dL,
                ws, ws_bytes, grad, d_edit_grad, stream)


def ivrgs_render_backward_accumulate(g, d_edit_table, p, b, cams, n_views, lowpass, bg, d_final_T, d_last, d_dL,
                                     ws, ws_bytes, grad, d_edit_grad, stream):
    return call("ivrgs_render_backward_accumulate", g, d_edit_table, p, b, cams, n_views, lowpass, bg, d_final_T,
                d_last, d_dL, ws, ws_bytes, grad, d_edit_grad, stream)


def ivrgs_render_backward_static(g, d_edit_table, p, b, cams, n_views, lowpass, bg, d_final_T, d_last, d_dL, grad,
                                 d_edit_grad, stream, allow=(IVRGS_OK,)):
    return call("ivrgs_render_backward_static", g, d_edit_table, p, b, cams, n_views, lowpass, bg, d_final_T,
                d_last, d_dL, grad, d_edit_grad, stream, allow=allow)


IVRGS_STATIC_SCRATCH_BYTES = 32 << 20


def ivrgs_set_option(name: str, value: int):
    return call("ivrgs_set_option", name.encode(), int(value))


def ivrgs_get_option(name: str) -> int:
    v = C.c_int64(0)
    call("ivrgs_get_option", name.encode(), C.byref(v))
    return int(v.value)


def prof_enable(on: bool):
    lib().ivrgs_prof_enable(1 if on else 0)


def prof_report() -> dict:
    """{kernel: (launches, total_ms)} since the previous report (synchronises)."""
    n = lib().ivrgs_prof_report(None, 0)
    buf = C.create_string_buffer(int(n) + 1)
    lib().ivrgs_prof_report(buf, int(n) + 1)
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms = line.split()
        out[name] = (int(cnt), float(ms))
    return out


def ivrgs_image_loss_workspace(cams, n_views) -> int:
    b = C.c_size_t(0)
    call("ivrgs_image_loss_workspace", cams, n_views, C.byref(b))
    return int(b.value)


def ivrgs_image_loss(d_rgba, d_target, cams, n_views, lambda_ssim, ws, ws_bytes, d_loss, d_dL, stream):
    return call("ivrgs_image_loss", d_rgba, d_target, cams, n_views, lambda_ssim, ws, ws_bytes, d_loss, d_dL, stream)


def ivrgs_edit_adam_init(d_table, n_models, d_state, stream):
    return call("ivrgs_edit_adam_init", d_table, n_models, d_state, stream)


def ivrgs_edit_adam(d_table, d_egrad, n_models, d_state, learn, lr, beta1, beta2, eps, stream):
    return call("ivrgs_edit_adam", d_table, d_egrad, n_models, d_state, learn, lr, beta1, beta2, eps, stream)


def ivrgs_render_aux(g, d_edit_table, p, b, cams, n_views, d_aux, stream):
    return call("ivrgs_render_aux", g, d_edit_table, p, b, cams, n_views, d_aux, stream)


def ivrgs_vq_build_workspace(n_models, k) -> int:
    b = C.c_size_t(0)
    call("ivrgs_vq_build_workspace", n_models, k, C.byref(b))
    return int(b.value)


def ivrgs_vq_build(src, k, iters, out, ws, ws_bytes, stream):
    return call("ivrgs_vq_build", src, k, iters, out, ws, ws_bytes, stream)

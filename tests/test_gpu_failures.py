"""Failure detection without a GPU fault.

The radix sort's look-back waits are bounded. A host-side injection makes the first radix
tile of every pass skip publishing its counts, so its successors' waits run out (after a short
bound) and the call reports IVRGS_ERR_TIMEOUT; nothing traps or hangs, every access stays in
bounds, and the next normal call on the same context is exact again. Host-side argument
errors and capacity errors are reported as status codes.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
import scenegen as sg
from paper_2504_17954_gb300 import Rasterizer
from paper_2504_17954_gb300 import _native as N
from paper_2504_17954_gb300.rasterizer import _stream, _vp
from tests import _gpu

pytestmark = pytest.mark.gpu


def _records(sizes, n, seed):
    xy, rad, depth = sg.synthetic_projected(sizes, n, seed)
    cams = [sg.look_at([3, 0, 0], W, H) for (W, H) in sizes]
    rast = Rasterizer(cams, n, 1, cull=False)  # records without conics: the rectangle lists
    rast.xy.copy_(torch.as_tensor(xy.reshape(-1, 2)))
    rast.radius.copy_(torch.as_tensor(rad.reshape(-1)))
    d = np.zeros((len(sizes) * n, 4), np.float32)
    d[:, 3] = depth.reshape(-1)
    rast.rgbd.copy_(torch.as_tensor(d))
    return rast, (xy, rad, depth)


@pytest.mark.parametrize("early", [0, 1])
def test_lookback_timeout_is_reported_and_context_survives(early):
    sizes = [(256, 256)]
    rast, (xy, rad, depth) = _records(sizes, 20000, 8)
    rast.bin("exact")  # sizes the buffers
    torch.cuda.synchronize()
    L = N.lib()
    old_scan, old_early = N.ivrgs_get_option("sort_scan"), N.ivrgs_get_option("sort_early")
    N.ivrgs_set_option("sort_scan", 0)  # the passes with device-side waits
    N.ivrgs_set_option("sort_early", early)  # counts published after or before the ranking
    L.ivrgs_debug_bin_hooks(2000, 0)
    try:
        p, b = rast.projected_struct(), rast.bins_struct()
        st = N.ivrgs_bin(C.byref(p), rast.cam_arr, rast.V, N.IVRGS_BIN_EXACT, _vp(rast.ws_bin), rast.ws_bin_bytes,
                         C.byref(b), _stream(), allow=(N.IVRGS_OK, N.IVRGS_ERR_TIMEOUT))
        assert st == N.IVRGS_ERR_TIMEOUT, N.last_error()
        assert "bound" in N.last_error()
        assert N.ivrgs_bin_check(_vp(rast.ws_bin), _stream(), allow=(N.IVRGS_ERR_TIMEOUT,)) == N.IVRGS_ERR_TIMEOUT
    finally:
        L.ivrgs_debug_bin_hooks(0, -1)
        N.ivrgs_set_option("sort_scan", old_scan)
        N.ivrgs_set_option("sort_early", old_early)
    # the context is healthy: a normal call is exact again and the flag is cleared
    rast.bin("exact")
    torch.cuda.synchronize()
    assert N.ivrgs_bin_check(_vp(rast.ws_bin), _stream()) == N.IVRGS_OK
    ref = oracle.bin_pairs(xy, rad, depth, sizes)
    k, v, r = _gpu.gpu_keys(rast)
    np.testing.assert_array_equal(k, ref.keys)
    np.testing.assert_array_equal(v, ref.values)


def test_status_codes_for_bad_calls():
    sizes = [(64, 64)]
    rast, _ = _records(sizes, 1000, 9)
    p, b = rast.projected_struct(), rast.bins_struct()
    # workspace too small
    st = N.ivrgs_bin(C.byref(p), rast.cam_arr, rast.V, N.IVRGS_BIN_EXACT, _vp(rast.ws_bin), 16, C.byref(b), _stream(),
                     allow=(N.IVRGS_ERR_CAPACITY,))
    assert st == N.IVRGS_ERR_CAPACITY and "workspace" in N.last_error()
    # wrong tile count in the bins struct
    b.n_tiles += 1
    st = N.ivrgs_bin(C.byref(p), rast.cam_arr, rast.V, N.IVRGS_BIN_EXACT, _vp(rast.ws_bin), rast.ws_bin_bytes,
                     C.byref(b), _stream(), allow=(N.IVRGS_ERR_INVALID_ARG,))
    assert st == N.IVRGS_ERR_INVALID_ARG
    # misaligned projected arrays
    b = rast.bins_struct()
    p.conic_o += 4
    st = N.call("ivrgs_render", C.byref(p), C.byref(b), rast.cam_arr, rast.V, rast.bg, _vp(rast.rgba),
                _vp(rast.final_T), _vp(rast.last), _stream(), allow=(N.IVRGS_ERR_INVALID_ARG,))
    assert st == N.IVRGS_ERR_INVALID_ARG and "misaligned" in N.last_error()
    # exact mode with a too-small pair buffer reports the required count
    p = rast.projected_struct()
    b = rast.bins_struct()
    b.capacity = 10
    st = N.ivrgs_bin(C.byref(p), rast.cam_arr, rast.V, N.IVRGS_BIN_EXACT, _vp(rast.ws_bin), rast.ws_bin_bytes,
                     C.byref(b), _stream(), allow=(N.IVRGS_ERR_CAPACITY,))
    assert st == N.IVRGS_ERR_CAPACITY and b.n_pairs > 10

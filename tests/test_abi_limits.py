"""Host-side size limits of the C ABI, checked without a GPU (the library validates before any
device work): at most IVRGS_MAX_VIEWS views per call, fewer than 2^30 records (n * views) and
pairs per binning call (the radix look-back carries 30-bit counts), and the workspace of the
largest allowed call is sized without overflow."""
import ctypes as C

import scenegen as sg
from paper_2504_17954_gb300 import _native as N
from paper_2504_17954_gb300.rasterizer import camera_structs


def _ws(n, cams, cap):
    arr, _ = camera_structs(cams)
    b = C.c_size_t(0)
    st = N.lib().ivrgs_bin_workspace(C.c_int64(n), C.c_int32(len(cams)), arr, C.c_int32(16), C.c_int32(16),
                                     C.c_int64(cap), C.byref(b))
    return st, b.value, N.lib().ivrgs_last_error().decode()


def test_record_limit():
    cams = [sg.look_at([3, 0, 0], 64, 64), sg.look_at([0, 3, 0], 64, 64)]
    st, _, msg = _ws(1 << 29, cams, 1024)  # 2^30 records
    assert st == N.IVRGS_ERR_INVALID_ARG and "2^30" in msg
    st, nbytes, _ = _ws((1 << 29) - 1, cams, 1024)  # the largest allowed
    assert st == N.IVRGS_OK and nbytes > 57 * ((1 << 30) - 2)  # ~57 bytes per record


def test_pair_capacity_limit():
    cams = [sg.look_at([3, 0, 0], 64, 64)]
    st, _, _ = _ws(1000, cams, N.IVRGS_MAX_PAIRS)
    assert st == N.IVRGS_ERR_INVALID_ARG
    st, nbytes, _ = _ws(1000, cams, N.IVRGS_MAX_PAIRS - 1)
    assert st == N.IVRGS_OK and nbytes > 8 * (N.IVRGS_MAX_PAIRS - 1)  # the pair ping-pong buffers alone


def test_view_limit():
    st, _, msg = _ws(10, [sg.look_at([3, 0, 0], 16, 16)] * (N.IVRGS_MAX_VIEWS + 1), 64)
    assert st == N.IVRGS_ERR_INVALID_ARG and "n_views" in msg
    st, _, _ = _ws(10, [sg.look_at([3, 0, 0], 16, 16)] * N.IVRGS_MAX_VIEWS, 64)
    assert st == N.IVRGS_OK


def test_empty_and_negative_sizes():
    """Zero Gaussians and zero pair capacity are valid (an empty scene sizes a small
    workspace); negative sizes are refused before any device work."""
    cams = [sg.look_at([3, 0, 0], 64, 64)]
    st, nbytes, _ = _ws(0, cams, 0)
    assert st == N.IVRGS_OK and nbytes > 0
    st, _, msg = _ws(-1, cams, 0)
    assert st == N.IVRGS_ERR_INVALID_ARG and "bad n" in msg
    st, _, msg = _ws(10, cams, -5)
    assert st == N.IVRGS_ERR_INVALID_ARG and "capacity" in msg
    b = C.c_size_t(0)
    assert N.lib().ivrgs_render_backward_workspace(C.c_int64(0), C.c_int32(1), C.byref(b)) == N.IVRGS_OK
    assert N.lib().ivrgs_render_backward_workspace(C.c_int64(-1), C.c_int32(1), C.byref(b)) == N.IVRGS_ERR_INVALID_ARG

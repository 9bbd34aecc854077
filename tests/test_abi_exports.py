"""The C-ABI library builds for sm_103a, loads without a GPU, exports every entry point
include/ivrgs.h declares, and rejects bad arguments on the host before touching the device."""
import ctypes as C
import shutil

import pytest

from paper_2504_17954_gb300 import _native as N


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") or __import__("os").path.exists("/usr/local/cuda/bin/nvcc"):
        from paper_2504_17954_gb300 import build
        build.build()
    return N.lib()


def test_every_declared_symbol_is_exported(lib):
    syms = N.declared_symbols()
    assert {"ivrgs_compose_edit", "ivrgs_project", "ivrgs_bin", "ivrgs_render", "ivrgs_render_backward"} <= set(syms)
    for s in syms:
        assert hasattr(lib, s), s


def test_host_side_argument_checks(lib):
    assert lib.ivrgs_version() >= 100
    assert lib.ivrgs_edit_table_floats(5) == 52
    st = lib.ivrgs_project(None, None, None, 1, 0.3, None, None)
    assert st == N.IVRGS_ERR_INVALID_ARG and "NULL" in N.last_error()
    cams = (N.ivrgs_camera * 2)()
    for c in cams:
        c.W = c.H = 32
        c.fx = c.fy = 40.0
        c.headlight = 1
    cams[1].pix_offset = 100  # overlaps view 0 (1024 pixels)
    b = C.c_size_t(0)
    st = lib.ivrgs_bin_workspace(10, 2, cams, 16, 16, 1000, C.byref(b))
    assert st == N.IVRGS_ERR_INVALID_ARG and "overlap" in N.last_error()
    cams[1].pix_offset = 1024
    assert lib.ivrgs_bin_workspace(10, 2, cams, 16, 16, 1000, C.byref(b)) == N.IVRGS_OK and b.value > 0
    assert lib.ivrgs_bin_workspace(10, 2, cams, 16, 8, 1000, C.byref(b)) == N.IVRGS_OK and b.value > 0
    for tw, th in ((8, 8), (16, 32), (16, 4), (32, 16)):  # tiles are 16 wide and 16 or 8 high
        assert lib.ivrgs_bin_workspace(10, 2, cams, tw, th, 1000, C.byref(b)) == N.IVRGS_ERR_UNSUPPORTED
    assert lib.ivrgs_bin_workspace(10, 0, cams, 16, 16, 1000, C.byref(b)) == N.IVRGS_ERR_INVALID_ARG
    assert lib.ivrgs_bin_workspace(10, 2, cams, 16, 16, 1 << 30, C.byref(b)) == N.IVRGS_ERR_INVALID_ARG
    cams[0].headlight = 0  # orbital light with a zero direction
    assert lib.ivrgs_bin_workspace(10, 2, cams, 16, 16, 1000, C.byref(b)) == N.IVRGS_ERR_INVALID_ARG
    assert lib.ivrgs_render_backward_workspace(10, 2, C.byref(b)) == N.IVRGS_OK and b.value >= 10 * 2 * 36
    # the auxiliary maps' reverse mode: 36 bytes of 2D-quantity gradients and 48 of value gradients
    # per (view, Gaussian); NULL arguments are refused before any device work
    assert lib.ivrgs_render_aux_backward_workspace(10, 2, C.byref(b)) == N.IVRGS_OK and b.value >= 10 * 2 * 84
    assert lib.ivrgs_render_aux_backward_workspace(-1, 2, C.byref(b)) == N.IVRGS_ERR_INVALID_ARG
    assert lib.ivrgs_render_aux_backward_workspace(10, 0, C.byref(b)) == N.IVRGS_ERR_INVALID_ARG
    st = lib.ivrgs_render_aux_backward(None, None, None, None, cams, 2, C.c_float(0.3), None, None, None, None,
                                       C.c_size_t(0), None, None, None)
    assert st == N.IVRGS_ERR_INVALID_ARG
    ed = (N.ivrgs_model_edit * 1)()
    li = N.ivrgs_light()
    assert lib.ivrgs_compose_edit(None, 0, ed, C.byref(li), None, None, None) == N.IVRGS_ERR_INVALID_ARG


def test_product_does_not_import_oracle():
    import pathlib
    root = pathlib.Path(N.__file__).parent
    for p in list(root.glob("*.py")) + list(root.glob("csrc/*")):
        text = p.read_text()
        assert "import oracle" not in text and "from oracle" not in text and "ivrgs_oracle" not in text, p


def test_header_constants_match_binding():
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "ivrgs.h")).read()
    pairs = re.findall(r"\b(IVRGS_[A-Z0-9_]+)\s*=\s*(\d+)", hdr)
    pairs += re.findall(r"#define\s+(IVRGS_[A-Z0-9_]+)\s+\(?(\d+)", hdr)
    checked = 0
    for name, val in pairs:
        if hasattr(N, name):
            assert getattr(N, name) == int(val), name
            checked += 1
    assert checked >= 8 and N.IVRGS_BIN_CULL == 2


def test_option_table_matches_the_autotuner_space(lib):
    """Every launch-shape option the autotuner searches is accepted by the library with every
    value in its range (set, read back, restored); out-of-range values and unknown names are
    refused with IVRGS_ERR_INVALID_ARG and leave the option unchanged. Host state only."""
    from paper_2504_17954_gb300.autotune import SPACE
    for name, values in SPACE.items():
        old = N.ivrgs_get_option(name)
        try:
            for v in values:
                N.ivrgs_set_option(name, v)
                assert N.ivrgs_get_option(name) == v, (name, v)
            for bad in (-1, max(values) + 1, 3 if 3 not in values else 16):
                st = lib.ivrgs_set_option(name.encode(), C.c_int64(bad))
                assert st == N.IVRGS_ERR_INVALID_ARG, (name, bad)
                assert N.ivrgs_get_option(name) == values[-1], (name, bad)
        finally:
            N.ivrgs_set_option(name, old)
    assert lib.ivrgs_set_option(b"no_such_option", C.c_int64(1)) == N.IVRGS_ERR_INVALID_ARG
    v = C.c_int64(0)
    assert lib.ivrgs_get_option(b"no_such_option", C.byref(v)) == N.IVRGS_ERR_INVALID_ARG

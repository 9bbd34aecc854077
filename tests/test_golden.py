"""The oracle against its regression record ``tests/golden/oracle_two_models_40x24.json``.

The record (written by ``tests/golden/make_golden.py`` through ``oracle/`` alone) holds one
small composed scene and the oracle's results for it. Two kinds of check:

* properties of the record that hold whatever the arithmetic (the runs partition the pairs;
  each tile's list is exactly the live Gaussians whose float32 tile rectangle holds the tile,
  rebuilt here by brute force from the record's own (u, v), radius and depth, ordered by
  depth bits then index; alpha in [0, 1]): a record that breaks one was written wrong;
* the oracle recomputes the record: ints exactly, floats to 1e-12 relative (the libm of the
  machine may round exp/log/pow differently in the last place). A failure means the oracle's
  arithmetic changed; the change has to name the passage of the paper that justifies it, and
  the record is then re-written by the script.
"""
import importlib.util
import json
import os

import numpy as np
import pytest

import oracle

_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
_spec = importlib.util.spec_from_file_location("make_golden", os.path.join(_DIR, "make_golden.py"))
mg = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(mg)

REL = 1e-12


@pytest.fixture(scope="module")
def rec():
    with open(os.path.join(_DIR, mg.NAME)) as f:
        return json.load(f)


def _close(got, want, what):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    assert got.shape == want.shape, what
    scale = max(1.0, float(np.abs(want).max(initial=0.0)))
    err = float(np.abs(got - want).max(initial=0.0))
    assert err <= REL * scale, f"{what}: max |diff| {err:.3e} (scale {scale:.3e})"


def test_inputs_round_trip_exactly(rec):
    w = mg.workload_from(rec["inputs"])
    assert mg.inputs_json(w) == rec["inputs"]
    assert w.n_gaussians == 16 and len(w.cameras) == 2


def test_record_is_a_valid_tiling(rec):
    out = rec["outputs"]
    cams = rec["inputs"]["cameras"]
    ranges = np.asarray(out["ranges"], np.int64)
    vals = np.asarray(out["values"], np.int64)
    toff = out["tile_offset"]
    # every pair in exactly one tile's run; runs laid out in tile order
    nz = ranges[ranges[:, 1] > ranges[:, 0]]
    assert nz[0, 0] == 0 and nz[-1, 1] == len(vals)
    assert np.array_equal(nz[1:, 0], nz[:-1, 1])
    for v, c in enumerate(cams):
        W, H = c["W"], c["H"]
        gx, gy = (W + 15) // 16, (H + 15) // 16
        assert toff[v + 1] - toff[v] == gx * gy
        view = out["views"][v]
        uv = np.asarray(view["uv32"], np.float32)
        rad = np.asarray(view["radius"])
        d32 = np.asarray(view["depth32"], np.float32)
        # rebuild every tile's list by brute force from the record's float32 decision inputs:
        # the half-open rectangle floor((u -+ r) / 16) (+1), clamped to the grid, in float32;
        # each list ordered by (depth bits, index)
        lists = [[] for _ in range(gx * gy)]
        for i in np.argsort(d32.view(np.uint32), kind="stable"):
            if rad[i] <= 0:
                continue
            r = np.float32(rad[i])
            rect = [np.floor((uv[i, 0] - r) / np.float32(16)), np.floor((uv[i, 0] + r) / np.float32(16)) + 1,
                    np.floor((uv[i, 1] - r) / np.float32(16)), np.floor((uv[i, 1] + r) / np.float32(16)) + 1]
            x0, x1 = (int(min(max(q, 0), gx)) for q in rect[:2])
            y0, y1 = (int(min(max(q, 0), gy)) for q in rect[2:])
            for ty in range(y0, y1):
                for tx in range(x0, x1):
                    lists[ty * gx + tx].append(int(i))
        for t in range(gx * gy):
            a, b = ranges[toff[v] + t]
            assert vals[a:b].tolist() == lists[t], (v, t)
        rgba = np.asarray(view["rgba"])
        assert np.all((rgba[:, 3] >= 0.0) & (rgba[:, 3] <= 1.0))
        assert 0.0 < view["rgba_sum"][3] <= W * H


def test_oracle_reproduces_the_record(rec):
    w = mg.workload_from(rec["inputs"])
    got = mg.outputs(w)
    want = rec["outputs"]
    for k in ("tile_offset", "ranges", "values"):
        assert got[k] == want[k], k
    for v, (gv, wv) in enumerate(zip(got["views"], want["views"])):
        for k in ("radius", "pixels", "last", "near_tie"):
            assert gv[k] == wv[k], (v, k)
        assert gv["depth32"] == wv["depth32"] and gv["uv32"] == wv["uv32"], v
        _close(gv["rgba"], wv["rgba"], f"view {v} rgba")
        _close(gv["rgba_sum"], wv["rgba_sum"], f"view {v} rgba_sum")
    for k in oracle.PARAMS:
        _close(got["grad"][k], want["grad"][k], f"grad {k}")
    _close(got["grad_edit"], want["grad_edit"], "grad_edit")
    _close(got["grad_light"], want["grad_light"], "grad_light")


def test_record_reacts_to_a_planted_change(rec):
    """The comparison is sharp enough to see a small change of an input (a stand-in for a
    changed step of the arithmetic): one Gaussian's opacity logit moved by 1e-6."""
    inp = json.loads(json.dumps(rec["inputs"]))
    m = inp["models"][0]
    m["opacity_logit"][3] = float(np.float32(m["opacity_logit"][3] + 1e-6))
    got = mg.outputs(mg.workload_from(inp))
    with pytest.raises(AssertionError):
        for v in range(2):
            _close(got["views"][v]["rgba_sum"], rec["outputs"]["views"][v]["rgba_sum"], "rgba_sum")
        _close(got["grad"]["mean"], rec["outputs"]["grad"]["mean"], "grad mean")

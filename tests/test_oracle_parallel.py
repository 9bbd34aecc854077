"""The all-core oracle driver (oracle/parallel.py) against the single-threaded oracle: the same
C routines over ranges of Gaussians, tile-row bands and tiles, so the sorted pairs, the image,
final T, last contributors and decision margins are bit for bit the same, and the gradients (per-thread sums added at the
end) agree to float64 rounding."""
import numpy as np

import oracle
import scenegen as sg
from oracle import parallel


def test_parallel_oracle_equals_the_serial_one():
    w = sg.tiny_scene(1500, 72, 56, 91, log_scale_mu=-3.2, n_models=3)
    cam = sg.look_at(3.0 * sg.random_direction(np.random.default_rng(92)), 72, 56, headlight=False,
                     light_dir=sg.orbital_light(30.0, 0.4))
    comp = oracle.compose(w.models)
    table = oracle.edit_table(w.edits)
    bg = np.array([0.1, 0.2, 0.3])
    ref = oracle.render(w.models, w.edits, [cam], bg=bg, comp=comp, table=table)
    rgba, T, last, mg, p, bins = parallel.render_view_parallel(comp, table, cam, bg, threads=5)
    np.testing.assert_array_equal(rgba, ref.images[0])
    np.testing.assert_array_equal(T, ref.final_T[0])
    np.testing.assert_array_equal(last, ref.last[0])
    np.testing.assert_array_equal(mg, ref.margins[0])
    np.testing.assert_array_equal(bins.keys, ref.bins.keys)
    np.testing.assert_array_equal(bins.values, ref.bins.values)
    np.testing.assert_array_equal(bins.ranges, ref.bins.ranges)
    dl = np.random.default_rng(93).normal(0, 1, (cam.H, cam.W, 4))
    gref = oracle.render_backward(ref, [cam], [dl], bg=bg)
    params, dedit, dlight = parallel.render_backward_view_parallel(comp, table, cam, p, bins, dl, bg, threads=5)
    for k in oracle.PARAMS:
        scale = max(1e-300, float(np.abs(gref.params[k]).max()))
        assert np.abs(params[k] - gref.params[k]).max() <= 1e-12 * scale, k
    np.testing.assert_allclose(dedit, gref.edit, rtol=1e-12, atol=1e-12 * np.abs(gref.edit).max())
    np.testing.assert_allclose(dlight, gref.light[0], rtol=1e-12, atol=1e-12 * np.abs(gref.light[0]).max())
    assert np.abs(gref.light[0]).max() > 0

"""The seeded input generators (scenegen: random draws and camera definitions, none of the
method's arithmetic) are deterministic and follow the stated recipe: each basic model's points
lie in its band of the blob field, the bands of composed scenes are disjoint, attribute arrays
are float32 with unit quaternions and normals, and the benchmark workloads have the stated
sizes."""

import numpy as np
import pytest

import scenegen as sg


@pytest.fixture(autouse=True)
def _no_cache(monkeypatch):
    monkeypatch.delenv("IVRGS_SCENE_CACHE", raising=False)


def _same(a, b):
    return all(np.array_equal(getattr(x, k), getattr(y, k)) for x, y in zip(a.models, b.models)
               for k in sg.ATTRS + ("palette",))


def test_seeded_and_deterministic():
    assert _same(sg.config1(), sg.config1())
    assert not _same(sg.config1(0), sg.config1(1))
    a, b = sg.tiny_scene(50, 32, 32, 5, n_models=2), sg.tiny_scene(50, 32, 32, 5, n_models=2)
    assert _same(a, b) and np.array_equal(a.cameras[0].R, b.cameras[0].R)


def test_band_sampling_and_attribute_recipe():
    f = sg.blob_field(8, 0)
    bands = sg.equal_bands(3)
    assert all(bands[i][1] == pytest.approx(bands[i + 1][0]) for i in range(2))
    models = sg.make_models(8, bands, [3000, 3000, 3000], 0)
    for (lo, hi), m in zip(bands, models):
        v = f(m.mean.astype(np.float64))
        # float32 storage of the positions moves the field value by far less than 1e-5
        assert np.all((v >= lo - 1e-5) & (v <= hi + 1e-5)), (lo, hi)
        for k in sg.ATTRS:
            assert getattr(m, k).dtype == np.float32, k
        np.testing.assert_allclose(np.linalg.norm(m.quat, axis=1), 1.0, atol=1e-6)
        np.testing.assert_allclose(np.linalg.norm(m.normal, axis=1), 1.0, atol=1e-6)
        np.testing.assert_allclose(m.dcolor.mean(0), 0.0, atol=1e-6)  # c_p is the mean albedo
        assert np.all(np.abs(m.mean) <= 1.0)


def test_camera_looks_at_the_target():
    cam = sg.look_at([0.0, -3.0, 1.0], 64, 48)
    R = cam.R.reshape(3, 3).astype(np.float64)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-6)
    xc = R @ np.zeros(3) + cam.t  # the target (origin) sits on the optical axis, in front
    assert abs(xc[0]) < 1e-5 and abs(xc[1]) < 1e-5 and xc[2] == pytest.approx(np.sqrt(10.0), rel=1e-6)
    assert (cam.cx, cam.cy) == (32.0, 24.0)


def test_benchmark_workload_sizes():
    w = sg.config4()
    assert w.n_gaussians == 1_000_000 and len(w.models) == 4 and len(w.cameras) == 8
    assert [m.n for m in w.models] == [100_000, 200_000, 300_000, 400_000]
    assert w.n_pixels == 6_653_952
    w1 = sg.config1()
    assert w1.n_gaussians == 10_000 and w1.n_pixels == 128 * 128

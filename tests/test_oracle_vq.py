"""Pins of the vector-quantisation oracle (oracle/vq.py, Sec. 4.4).

* Separated clusters: with k equal to their number, Lloyd ends at the cluster means.
* Lloyd never increases the quantisation error (per iteration), and with k at least the
  number of distinct values spaced evenly, every value is reproduced exactly.
* Nearest-centroid rule: brute force over all centroids, ties to the lower index.
* Round trip: decode(build()) gives every component its nearest codebook value of its model.
"""
import numpy as np

from oracle import vq


def test_separated_clusters_end_at_their_means():
    rng = np.random.default_rng(1)
    centres = np.array([-2.0, 0.5, 1.0, 3.0])
    v = np.concatenate([c + rng.normal(0, 0.01, 200) for c in centres])
    cent = vq.kmeans_1d(v, 4, 20)
    means = [v[i * 200:(i + 1) * 200].mean() for i in range(4)]
    np.testing.assert_allclose(cent, means, rtol=0, atol=1e-12)


def test_lloyd_is_monotone_and_exact_on_few_values():
    rng = np.random.default_rng(2)
    v = rng.normal(0, 1, 5000) ** 3
    err = []
    for it in range(8):
        c = vq.kmeans_1d(v, 16, it)
        err.append(((c[vq.nearest(c, v)] - v) ** 2).mean())
    assert all(b <= a + 1e-15 for a, b in zip(err, err[1:])), err
    vals = np.linspace(-1, 1, 7)
    w = rng.choice(vals, 1000)
    c = vq.kmeans_1d(w, 7, 3)
    np.testing.assert_allclose(c[vq.nearest(c, w)], w, rtol=0, atol=1e-12)


def test_nearest_matches_brute_force():
    rng = np.random.default_rng(3)
    c = np.sort(rng.normal(0, 1, 33))
    v = rng.normal(0, 2, 4000)
    d = np.abs(v[:, None] - c[None, :])
    np.testing.assert_array_equal(vq.nearest(c, v), np.argmin(d, axis=1))
    # a value on the (computed) midpoint goes to the lower centroid
    mids = 0.5 * (c[:-1] + c[1:])
    np.testing.assert_array_equal(vq.nearest(c, mids), np.arange(len(mids)))
    np.testing.assert_array_equal(vq.nearest(c, np.nextafter(mids, np.inf)), np.arange(1, len(c)))


def test_build_decode_round_trip():
    rng = np.random.default_rng(4)
    n, M = 3000, 3
    mid = rng.integers(0, M, n)
    arrs = {"log_scale": rng.normal(-4, 0.5, (n, 3)), "quat": rng.normal(0, 1, (n, 4)),
            "opacity_logit": rng.normal(0, 1.5, n), "dcolor": rng.uniform(-0.2, 0.2, (n, 3)),
            "kads": np.c_[rng.uniform(0.1, 0.3, n), rng.uniform(0.5, 0.9, n), rng.uniform(0.2, 0.4, n),
                          rng.uniform(10, 50, n)]}
    cb, idx = vq.build(arrs, mid, M, 64, 6)
    dec = vq.decode(cb, idx, mid)
    for m in range(M):
        sel = mid == m
        for name, a in (("log_scale", 0), ("quat", 1), ("dcolor", 3)):
            vals = arrs[name][sel]
            d = np.abs(vals[..., None] - cb[m, a][None, None, :])
            np.testing.assert_array_equal(dec[name][sel], cb[m, a][np.argmin(d, -1)])
        for j in range(4):
            vals = arrs["kads"][sel, j]
            np.testing.assert_array_equal(dec["kads"][sel, j], cb[m, 4 + j][np.argmin(np.abs(vals[:, None] - cb[m, 4 + j]), 1)])
    # 64 levels of a smooth distribution: small relative error
    rel = np.abs(dec["kads"][:, 3] - arrs["kads"][:, 3]).max() / 40.0
    assert rel < 0.02
